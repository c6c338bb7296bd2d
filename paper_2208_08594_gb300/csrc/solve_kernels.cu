// Solve-phase kernels: BSR block-row kernels (SpMV / residual, decoupled pressure
// restriction, stage-N block GS, BILU(0) sweeps), scalar CSR level kernels (PGS-MC
// sweeps, residual + aggregate restriction, prolongation, dense coarsest GEMV) and the
// FP64 Krylov reductions.  All are memory-bound streaming kernels: one thread group of
// GP(b) lanes owns a block row, lane r owns equation r of the block and reads that row
// of every b x b block (b contiguous values), so a group reads whole blocks with
// 8/16-byte vector loads and consecutive groups read consecutive block rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace msp {

namespace {

constexpr int kThreads = 256;

template <int B>
struct Gp {
  static constexpr int v = B <= 1 ? 1 : (B <= 2 ? 2 : (B <= 4 ? 4 : 8));
};

// The level-0 block-row kernels are bound by chains of dependent loads per row (row
// pointers, column index, gathered x): launched with one thread (group) per row and as
// many blocks as that takes, the block scheduler refills SMs as blocks finish, where a
// grid-stride loop capped at one resident wave left SMs idle behind the threads that drew
// an extra row (stage-N colour of 561k rows: 81.9 against 94.2 us).
constexpr unsigned kRowGridPerSm = 1u << 20;

// Load B consecutive values with the widest aligned vector loads (rows start at
// multiples of B*sizeof(T) bytes from a 256-byte aligned allocation).  Components are
// assigned one by one: copying a loaded vector into the array as raw bytes would put
// the array in local memory.
template <int B, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&r)[B]) {
  if constexpr (sizeof(T) == 8 && B % 2 == 0) {
#pragma unroll
    for (int k = 0; k < B / 2; ++k) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p) + k);
      r[2 * k] = t.x;
      r[2 * k + 1] = t.y;
    }
  } else if constexpr (sizeof(T) == 4 && B % 4 == 0) {
#pragma unroll
    for (int k = 0; k < B / 4; ++k) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + k);
      r[4 * k] = t.x;
      r[4 * k + 1] = t.y;
      r[4 * k + 2] = t.z;
      r[4 * k + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 4 && B % 2 == 0) {
#pragma unroll
    for (int k = 0; k < B / 2; ++k) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(p) + k);
      r[2 * k] = t.x;
      r[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < B; ++c) r[c] = __ldg(p + c);
  }
}

// acc + a . x  (one FMA per product: FP64 FMA issue is the binding resource of the
// FP64 block kernels on GB300)
template <int B, typename T>
__device__ __forceinline__ T fma_row(const T (&a)[B], const T (&x)[B], T acc) {
#pragma unroll
  for (int c = 0; c < B; ++c) acc = fma(a[c], x[c], acc);
  return acc;
}

// acc - a . x
template <int B, typename T>
__device__ __forceinline__ T fnma_row(const T (&a)[B], const T (&x)[B], T acc) {
#pragma unroll
  for (int c = 0; c < B; ++c) acc = fma(-a[c], x[c], acc);
  return acc;
}

// sum over the GP lanes of a group (all lanes of the group participate)
template <int GP, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = GP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GP);
  return v;
}

// One long row by one thread block (kThreads threads): S_r = sum over the blocks q in
// [q0, q1), q != skip, of sum_c A_q[r][c] x_{ci[q]}[c], with A_q the R x C values at
// vals + q * R * C (row-major) and x_j the C values at x + j * xs + xo.  The block holds
// NB = kThreads / R blocks at a time, R threads each (thread t: row t % R of blocks
// q0 + t / R, q0 + t / R + NB, ...), the same few registers per thread as the lane-group
// kernels; thread r < R returns S_r, the partial sums combined through shared memory in
// a fixed order.  Every thread of the block calls it (it synchronises the block).  x rows
// are never written by the launch.
template <int R, int C, typename T>
__device__ __forceinline__ T block_row_sum(int q0, int q1, int skip, const int* __restrict__ ci,
                                           const T* __restrict__ vals, const T* x, int xs,
                                           int xo) {
  constexpr int NB = kThreads / R, G = 8;
  __shared__ T part_s[kThreads];
  __shared__ T group_s[G * 8];
  const int t = threadIdx.x;
  const int r = t % R, k0 = t / R;
  T part = T(0);
  if (k0 < NB) {
#pragma unroll 1
    for (int q = q0 + k0; q < q1; q += NB) {
      if (q == skip) continue;
      const T* xr = x + (size_t)__ldg(ci + q) * xs + xo;
      const T* a = vals + ((size_t)q * R + r) * C;
#pragma unroll
      for (int c = 0; c < C; ++c) part = fma(__ldg(a + c), __ldg(xr + c), part);
    }
  }
  part_s[t] = part;
  __syncthreads();
  if (t < R * G) {  // G partial sums per row r, then their sum in order
    const int rr = t % R, g = t / R;
    T sg = T(0);
    for (int k = g; k < NB; k += G) sg += part_s[rr + k * R];
    group_s[g * R + rr] = sg;
  }
  __syncthreads();
  T tot = T(0);
  if (t < R) {
#pragma unroll
    for (int g = 0; g < G; ++g) tot += group_s[g * R + t];
  }
  __syncthreads();  // the shared arrays are reused by the next row
  return tot;
}

// A colour made only of long rows (the well rows form one at level 0): one thread block
// per row, every thread of the block holding two of the row's blocks in the first pass,
// whose column indices and values it loads before `griddepcontrol.wait` (PDL: launched as
// a programmatic dependent of the previous colour's sweep, it waits only for the gathered
// x, which it reads from L2, where the previous kernel's writes are).  Thread r < R
// returns S_r (as block_row_sum, in a fixed order).
template <int R, int C, typename T, bool PDL>
__device__ __forceinline__ T long_colour_row_sum(int q0, int q1, int skip,
                                                 const int* __restrict__ ci,
                                                 const T* __restrict__ vals, const T* x, int xs,
                                                 int xo) {
  constexpr int NB = kThreads / R, G = 8;
  __shared__ T part_s[kThreads];
  __shared__ T group_s[G * 8];
  const int t = threadIdx.x;
  const int r = t % R, k0 = t / R;
  const int qa = q0 + k0, qb = q0 + k0 + NB;
  const bool ha = k0 < NB && qa < q1 && qa != skip;
  const bool hb = k0 < NB && qb < q1 && qb != skip;
  const int ja = ha ? __ldg(ci + qa) : 0, jb = hb ? __ldg(ci + qb) : 0;
  T aa[C], ab[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    aa[c] = ha ? __ldg(vals + ((size_t)qa * R + r) * C + c) : T(0);
    ab[c] = hb ? __ldg(vals + ((size_t)qb * R + r) * C + c) : T(0);
  }
  if constexpr (PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
  T part = T(0);
  if (ha) {
#pragma unroll
    for (int c = 0; c < C; ++c) part = fma(aa[c], __ldcg(x + (size_t)ja * xs + xo + c), part);
  }
  if (hb) {
#pragma unroll
    for (int c = 0; c < C; ++c) part = fma(ab[c], __ldcg(x + (size_t)jb * xs + xo + c), part);
  }
  if (k0 < NB) {  // rows longer than 2 NB blocks
#pragma unroll 1
    for (int q = q0 + k0 + 2 * NB; q < q1; q += NB) {
      if (q == skip) continue;
      const T* xr = x + (size_t)__ldg(ci + q) * xs + xo;
      const T* a = vals + ((size_t)q * R + r) * C;
#pragma unroll
      for (int c = 0; c < C; ++c) part = fma(__ldg(a + c), __ldcg(xr + c), part);
    }
  }
  part_s[t] = part;
  __syncthreads();
  if (t < R * G) {
    const int rr = t % R, g = t / R;
    T sg = T(0);
    for (int k = g; k < NB; k += G) sg += part_s[rr + k * R];
    group_s[g * R + rr] = sg;
  }
  __syncthreads();
  T tot = T(0);
  if (t < R) {
#pragma unroll
    for (int g = 0; g < G; ++g) tot += group_s[g * R + t];
  }
  return tot;
}

// stage-N sweep over a colour of long rows only: block q takes row r0 + q
template <int B, typename T, bool PDL>
__global__ void __launch_bounds__(kThreads) bgs_long_colour_kernel(
    int r0, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ dpos,
    const T* __restrict__ aN, const T* __restrict__ y, T* __restrict__ w, bool lower_only,
    bool zero_pressure, const unsigned char* __restrict__ rmask) {
  constexpr int BN = B - 1;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int i = r0 + blockIdx.x;
  if (rmask && !rmask[i]) return;  // uniform over the block
  const int pd = __ldg(dpos + i);
  const int l = threadIdx.x;
  const T yl = l < BN ? __ldg(y + (size_t)i * BN + l) : T(0);
  const T sl = long_colour_row_sum<BN, BN, T, PDL>(__ldg(rp + i), lower_only ? pd : __ldg(rp + i + 1),
                                                   pd, ci, aN, w, B, 1);
  if (l < BN) w[(size_t)i * B + 1 + l] = yl - sl;
  if (zero_pressure && l == 0) w[(size_t)i * B] = T(0);
}

// BILU(0) forward over a colour of long rows only
template <int B, typename T, bool PDL>
__global__ void __launch_bounds__(kThreads) bilu_fwd_long_colour_kernel(
    int r0, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ dpos,
    const T* __restrict__ lu, const T* __restrict__ r, T* __restrict__ y,
    const unsigned char* __restrict__ rmask) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int i = r0 + blockIdx.x;
  if (rmask && !rmask[i]) return;
  const int l = threadIdx.x;
  const T rl = l < B ? __ldg(r + (size_t)i * B + l) : T(0);
  const T sl = long_colour_row_sum<B, B, T, PDL>(__ldg(rp + i), __ldg(dpos + i), -1, ci, lu, y, B, 0);
  if (l < B) y[(size_t)i * B + l] = rl - sl;
}

// BILU(0) backward over a colour of long rows only: x_i = U_ii^-1 (y_i - sum_{j>i} U_ij x_j)
template <int B, typename T, bool PDL>
__global__ void __launch_bounds__(kThreads) bilu_bwd_long_colour_kernel(
    int r0, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ dpos,
    const T* __restrict__ lu, const T* __restrict__ uinv, const T* __restrict__ y,
    T* __restrict__ x, T* __restrict__ w, const unsigned char* __restrict__ rmask) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int i = r0 + blockIdx.x;
  if (rmask && !rmask[i]) return;
  const int l = threadIdx.x;
  const T sl = long_colour_row_sum<B, B, T, PDL>(__ldg(dpos + i) + 1, __ldg(rp + i + 1), -1, ci, lu,
                                                 x, B, 0);
  if (l >= kWarp) return;  // the row's outputs are warp 0's
  const T t = l < B ? __ldcg(y + (size_t)i * B + l) - sl : T(0);
  const T* ui = uinv + ((size_t)i * B + (l < B ? l : 0)) * B;
  T out = T(0);
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const T tc = __shfl_sync(0xffffffffu, t, c);
    if (l < B) out = fma(__ldg(ui + c), tc, out);
  }
  if (l < B) {
    x[(size_t)i * B + l] = out;
    w[(size_t)i * B + l] += out;
  }
}

// blocks of a launch: enough for one thread per work item and one block per long row
inline unsigned with_long_rows(unsigned grid, int nlong) {
  return std::max(grid, (unsigned)std::min(nlong, 1 << 16));
}

// ----------------------------------------------------------------------------------
// y = A x  or  y = g - A x
// ----------------------------------------------------------------------------------
template <int B, typename T, bool RES>
__global__ void __launch_bounds__(kThreads) bsr_spmv_kernel(int nb, const int* __restrict__ rp,
                                                           const int* __restrict__ ci,
                                                           const T* __restrict__ v,
                                                           const T* __restrict__ x,
                                                           const T* __restrict__ g,
                                                           T* __restrict__ y,
                                                           const unsigned char* __restrict__ rmask,
                                                           const int* __restrict__ lrows,
                                                           int nlong, int lthr) {
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const T sl = block_row_sum<B, B>(__ldg(rp + i), __ldg(rp + i + 1), -1, ci, v, x, B, 0);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    if (l < B) y[(size_t)i * B + l] = RES ? g[(size_t)i * B + l] - sl : sl;
  }
  constexpr int GP = Gp<B>::v;
  const int lane = threadIdx.x % GP;
  const int gpb = blockDim.x / GP;
  const int stride = gridDim.x * gpb;
  for (int i = blockIdx.x * gpb + threadIdx.x / GP; i < nb; i += stride) {
    if (lane >= B || (rmask && !rmask[i])) continue;
    const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
    if (p1 - p0 > lthr) continue;  // taken by a block above
    T acc = RES ? g[(size_t)i * B + lane] : T(0);
    int p = p0;
    for (; p + 1 < p1; p += 2) {  // two blocks in flight
      const int j0 = __ldg(ci + p), j1 = __ldg(ci + p + 1);
      T a0[B], a1[B], x0[B], x1[B];
      load_row<B>(v + ((size_t)p * B + lane) * B, a0);
      load_row<B>(v + ((size_t)(p + 1) * B + lane) * B, a1);
      load_row<B>(x + (size_t)j0 * B, x0);
      load_row<B>(x + (size_t)j1 * B, x1);
      acc = RES ? fnma_row<B>(a0, x0, acc) : fma_row<B>(a0, x0, acc);
      acc = RES ? fnma_row<B>(a1, x1, acc) : fma_row<B>(a1, x1, acc);
    }
    if (p < p1) {
      const int j0 = __ldg(ci + p);
      T a0[B], x0[B];
      load_row<B>(v + ((size_t)p * B + lane) * B, a0);
      load_row<B>(x + (size_t)j0 * B, x0);
      acc = RES ? fnma_row<B>(a0, x0, acc) : fma_row<B>(a0, x0, acc);
    }
    y[(size_t)i * B + lane] = acc;
  }
}

// ----------------------------------------------------------------------------------
// rP[i] = omega_i^T (g_i - (A w)_i); with WR the residual g - A w is also stored in r
// ----------------------------------------------------------------------------------
template <int B, typename T, bool WR>
__global__ void __launch_bounds__(kThreads) bsr_restrict_p_kernel(
    int nb, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
    const T* __restrict__ w, const T* __restrict__ g, const T* __restrict__ omega,
    T* __restrict__ rP, T* __restrict__ r, const unsigned char* __restrict__ rmask,
    const int* __restrict__ lrows, int nlong, int lthr) {
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const T sl = block_row_sum<B, B>(__ldg(rp + i), __ldg(rp + i + 1), -1, ci, v, w, B, 0);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    T term = T(0);
    if (l < B) {
      const T al = g[(size_t)i * B + l] - sl;
      if (WR) r[(size_t)i * B + l] = al;
      term = omega ? al * omega[(size_t)i * B + l] : (l == 0 ? al : T(0));
    }
    T res = term;  // lane 0: the B terms in order
#pragma unroll
    for (int k = 1; k < B; ++k) res += __shfl_sync(0xffffffffu, term, k);
    if (l == 0) rP[i] = res;
  }
  constexpr int GP = Gp<B>::v;
  const int lane = threadIdx.x % GP;
  const int gpb = blockDim.x / GP;
  // the loop bound depends on the block only, so every lane reaches the group shuffle
  for (int base = blockIdx.x * gpb; base < nb; base += gridDim.x * gpb) {
    const int i = base + threadIdx.x / GP;
    T res = T(0);
    bool live = (i < nb) && (!rmask || rmask[i]);
    // rows taken by a block above: every lane of the group reads the same length
    if (live && __ldg(rp + i + 1) - __ldg(rp + i) > lthr) live = false;
    const bool active = live && (lane < B);
    if (active) {
      const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
      T acc = g[(size_t)i * B + lane];
      int p = p0;
      for (; p + 1 < p1; p += 2) {  // two blocks in flight, same order as one at a time
        const int j0 = __ldg(ci + p), j1 = __ldg(ci + p + 1);
        T a0[B], a1[B], x0[B], x1[B];
        load_row<B>(v + ((size_t)p * B + lane) * B, a0);
        load_row<B>(v + ((size_t)(p + 1) * B + lane) * B, a1);
        load_row<B>(w + (size_t)j0 * B, x0);
        load_row<B>(w + (size_t)j1 * B, x1);
        acc = fnma_row<B>(a0, x0, acc);
        acc = fnma_row<B>(a1, x1, acc);
      }
      if (p < p1) {
        const int j0 = __ldg(ci + p);
        T a0[B], x0[B];
        load_row<B>(v + ((size_t)p * B + lane) * B, a0);
        load_row<B>(w + (size_t)j0 * B, x0);
        acc = fnma_row<B>(a0, x0, acc);
      }
      if (WR) r[(size_t)i * B + lane] = acc;
      res = omega ? acc * omega[(size_t)i * B + lane] : (lane == 0 ? acc : T(0));
    }
    res = group_sum<GP>(res);
    if (live && lane == 0) rP[i] = res;
  }
}

// ----------------------------------------------------------------------------------
// Pressure correction of stage P applied to the residual as well as to w:
//   r_i <- r_i - sum_j A_ij[:, 0] e_j,   w_i[0] <- w_i[0] + e_i
// With r = g - A w on entry this leaves r = g - A (w + Pi_P e), the residual that stage R
// starts from, reading one column of each block (c0, b values per block) instead of
// the whole block.
// ----------------------------------------------------------------------------------
template <int B, typename T>
__global__ void __launch_bounds__(kThreads) bsr_col0_update_kernel(
    int nb, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ c0,
    const T* __restrict__ e, T* __restrict__ r, T* __restrict__ w,
    const unsigned char* __restrict__ rmask, const int* __restrict__ lrows, int nlong,
    int lthr) {
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const T sl = block_row_sum<B, 1>(__ldg(rp + i), __ldg(rp + i + 1), -1, ci, c0, e, 1, 0);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    if (l < B) r[(size_t)i * B + l] -= sl;
    if (l == 0) w[(size_t)i * B] += __ldg(e + i);
  }
  constexpr int GP = Gp<B>::v;
  const int lane = threadIdx.x % GP;
  const int gpb = blockDim.x / GP;
  const int stride = gridDim.x * gpb;
  for (int i = blockIdx.x * gpb + threadIdx.x / GP; i < nb; i += stride) {
    if (lane >= B || (rmask && !rmask[i])) continue;
    const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
    if (p1 - p0 > lthr) continue;  // taken by a block above
    T acc = r[(size_t)i * B + lane];
    int p = p0;
    for (; p + 3 < p1; p += 4) {  // four blocks in flight
      const int j0 = __ldg(ci + p), j1 = __ldg(ci + p + 1);
      const int j2 = __ldg(ci + p + 2), j3 = __ldg(ci + p + 3);
      const T a0 = __ldg(c0 + (size_t)p * B + lane), a1 = __ldg(c0 + (size_t)(p + 1) * B + lane);
      const T a2 = __ldg(c0 + (size_t)(p + 2) * B + lane), a3 = __ldg(c0 + (size_t)(p + 3) * B + lane);
      const T e0 = __ldg(e + j0), e1 = __ldg(e + j1), e2 = __ldg(e + j2), e3 = __ldg(e + j3);
      acc = fma(-a0, e0, acc);
      acc = fma(-a1, e1, acc);
      acc = fma(-a2, e2, acc);
      acc = fma(-a3, e3, acc);
    }
    for (; p < p1; ++p) acc = fma(-__ldg(c0 + (size_t)p * B + lane), __ldg(e + __ldg(ci + p)), acc);
    r[(size_t)i * B + lane] = acc;
    if (lane == 0) w[(size_t)i * B] += __ldg(e + i);
  }
}

// c0[p * b + r] = v[p * b * b + r * b]: column 0 (the pressure column) of every block
template <typename T>
__global__ void extract_col0_kernel(size_t nnzb, int b, const T* __restrict__ v,
                                    T* __restrict__ c0) {
  const size_t total = nnzb * (size_t)b;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x)
    c0[t] = v[t * b];
}

// ----------------------------------------------------------------------------------
// stage N block GS sweep over one colour (BN = b - 1 concentration unknowns)
// ----------------------------------------------------------------------------------
template <int B, typename T>
__global__ void __launch_bounds__(kThreads) bgs_colour_kernel(
    int r0, int r1, const int* __restrict__ rp, const int* __restrict__ ci,
    const int* __restrict__ dpos, const T* __restrict__ aN, const T* __restrict__ y,
    T* __restrict__ w, bool lower_only, bool zero_pressure,
    const unsigned char* __restrict__ rmask, const int* __restrict__ lrows, int nlong,
    int lthr) {
  constexpr int BN = B - 1;
  // a colour of long rows may follow as a programmatic dependent (it waits for this grid
  // before it reads w)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const int pd = __ldg(dpos + i);
    const T sl = block_row_sum<BN, BN>(__ldg(rp + i), lower_only ? pd : __ldg(rp + i + 1), pd,
                                      ci, aN, w, B, 1);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    if (l < BN) w[(size_t)i * B + 1 + l] = y[(size_t)i * BN + l] - sl;
    if (zero_pressure && l == 0) w[(size_t)i * B] = T(0);
  }
  // BN consecutive threads per row (thread t: row r0 + t / BN, sub-block row t % BN); a
  // row may straddle two warps, so every lane is busy whatever b is
  const size_t total = (size_t)(r1 - r0) * BN;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = r0 + (int)(t / BN), lane = (int)(t % BN);
    if (rmask && !rmask[i]) continue;
    T acc = y[(size_t)i * BN + lane];
    const int p0 = __ldg(rp + i), pd = __ldg(dpos + i), p1 = __ldg(rp + i + 1);
    if (p1 - p0 > lthr) continue;  // taken by a block above
    const int pend = lower_only ? pd : p1;
    // the off-diagonal blocks only (the diagonal block is not read): the k-th of them
    // sits at p0 + k, one further on from the diagonal position
    const int cnt = (pend - p0) - (pd < pend ? 1 : 0);
    auto at = [&](int k) { return p0 + k + (p0 + k >= pd ? 1 : 0); };
    // w rows of other colours: none of them is written by this launch
    auto load = [&](int p, T (&a)[BN], T (&xx)[BN]) {
      const T* xr = w + (size_t)__ldg(ci + p) * B + 1;
      const T* ar = aN + ((size_t)p * BN + lane) * BN;
#pragma unroll
      for (int c = 0; c < BN; ++c) {
        a[c] = __ldg(ar + c);
        xx[c] = __ldg(xr + c);
      }
    };
    int k = 0;
    for (; k + 1 < cnt; k += 2) {  // two blocks in flight, same order as one at a time
      T a0[BN], x0[BN], a1[BN], x1[BN];
      load(at(k), a0, x0);
      load(at(k + 1), a1, x1);
#pragma unroll
      for (int c = 0; c < BN; ++c) acc = fma(-a0[c], x0[c], acc);
#pragma unroll
      for (int c = 0; c < BN; ++c) acc = fma(-a1[c], x1[c], acc);
    }
    if (k < cnt) {
      T a0[BN], x0[BN];
      load(at(k), a0, x0);
#pragma unroll
      for (int c = 0; c < BN; ++c) acc = fma(-a0[c], x0[c], acc);
    }
    // the blocks are D_N,i^-1 A_ij and y_i = D_N,i^-1 g_i: acc is x_i itself
    w[(size_t)i * B + 1 + lane] = acc;
    if (zero_pressure && lane == 0) w[(size_t)i * B] = T(0);
  }
}

// y_i = D_N,i^-1 g_i (concentration part of g), once per stage-N application: the sweeps
// then start every row from y_i and use the pre-scaled blocks
template <int BN, typename T>
__global__ void nscale_kernel(int nb, const T* __restrict__ dNinv, const T* __restrict__ g,
                              T* __restrict__ y) {
  constexpr int B = BN + 1;
  const size_t total = (size_t)nb * BN;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / BN;  // row i, concentration unknown t % BN
    const T* d = dNinv + t * BN;
    const T* gi = g + i * B + 1;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < BN; ++c) acc = fma(__ldg(d + c), gi[c], acc);
    y[t] = acc;
  }
}

// ----------------------------------------------------------------------------------
// BILU(0) forward (unit lower) over one colour
// ----------------------------------------------------------------------------------
template <int B, typename T>
__global__ void __launch_bounds__(kThreads) bilu_fwd_kernel(
    int r0, int r1, const int* __restrict__ rp, const int* __restrict__ ci,
    const int* __restrict__ dpos, const T* __restrict__ lu, const T* __restrict__ r,
    T* __restrict__ y, const unsigned char* __restrict__ rmask, const int* __restrict__ lrows,
    int nlong, int lthr) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // as in the stage-N sweep
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const T sl = block_row_sum<B, B>(__ldg(rp + i), __ldg(dpos + i), -1, ci, lu, y, B, 0);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    if (l < B) y[(size_t)i * B + l] = r[(size_t)i * B + l] - sl;
  }
  constexpr int GP = Gp<B>::v;
  const int lane = threadIdx.x % GP;
  const int gpb = blockDim.x / GP;
  for (int i = r0 + blockIdx.x * gpb + threadIdx.x / GP; i < r1; i += gridDim.x * gpb) {
    if (lane >= B || (rmask && !rmask[i])) continue;
    if (__ldg(rp + i + 1) - __ldg(rp + i) > lthr) continue;  // taken by a block above
    T acc = r[(size_t)i * B + lane];
    const int p0 = __ldg(rp + i), pd = __ldg(dpos + i);
    // y rows of earlier colours: none of them is written by this launch
    int p = p0;
    for (; p + 1 < pd; p += 2) {  // two blocks in flight, same order as one at a time
      const int j0 = __ldg(ci + p), j1 = __ldg(ci + p + 1);
      T a0[B], a1[B], y0[B], y1[B];
      load_row<B>(lu + ((size_t)p * B + lane) * B, a0);
      load_row<B>(lu + ((size_t)(p + 1) * B + lane) * B, a1);
      load_row<B>(y + (size_t)j0 * B, y0);
      load_row<B>(y + (size_t)j1 * B, y1);
      acc = fnma_row<B>(a0, y0, acc);
      acc = fnma_row<B>(a1, y1, acc);
    }
    if (p < pd) {
      const int j0 = __ldg(ci + p);
      T a0[B], y0[B];
      load_row<B>(lu + ((size_t)p * B + lane) * B, a0);
      load_row<B>(y + (size_t)j0 * B, y0);
      acc = fnma_row<B>(a0, y0, acc);
    }
    y[(size_t)i * B + lane] = acc;
  }
}

// BILU(0) backward over one colour: x_i = U_ii^{-1} (y_i - sum_{j>i} U_ij x_j); w_i += x_i
template <int B, typename T>
__global__ void __launch_bounds__(kThreads) bilu_bwd_kernel(
    int r0, int r1, const int* __restrict__ rp, const int* __restrict__ ci,
    const int* __restrict__ dpos, const T* __restrict__ lu, const T* __restrict__ uinv,
    const T* __restrict__ y, T* __restrict__ x, T* __restrict__ w,
    const unsigned char* __restrict__ rmask, const int* __restrict__ lrows, int nlong,
    int lthr) {
  for (int q = blockIdx.x; q < nlong; q += gridDim.x) {  // long rows: a block each
    const int i = lrows[q];
    if (rmask && !rmask[i]) continue;
    const T sl = block_row_sum<B, B>(__ldg(dpos + i) + 1, __ldg(rp + i + 1), -1, ci, lu, x, B, 0);
    if (threadIdx.x >= kWarp) continue;  // the row's outputs are warp 0's
    const int l = threadIdx.x;
    const T t = l < B ? y[(size_t)i * B + l] - sl : T(0);
    const T* ui = uinv + ((size_t)i * B + (l < B ? l : 0)) * B;
    T out = T(0);
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const T tc = __shfl_sync(0xffffffffu, t, c);
      if (l < B) out = fma(__ldg(ui + c), tc, out);
    }
    if (l < B) {
      x[(size_t)i * B + l] = out;
      w[(size_t)i * B + l] += out;
    }
  }
  constexpr int GP = Gp<B>::v;
  const int lane = threadIdx.x % GP;
  const int gpb = blockDim.x / GP;
  const int grp = threadIdx.x / GP;
  for (int base = r0 + blockIdx.x * gpb; base < r1; base += gridDim.x * gpb) {
    const int i = base + grp;
    // rows taken by a block above are left out; every lane of the group reads the same length
    const bool active = (i < r1) && (lane < B) && (!rmask || rmask[i]) &&
                        __ldg(rp + i + 1) - __ldg(rp + i) <= lthr;
    T acc = T(0);
    if (active) {
      acc = y[(size_t)i * B + lane];
      const int pd = __ldg(dpos + i), p1 = __ldg(rp + i + 1);
      // x rows of later colours: none of them is written by this launch
      int p = pd + 1;
      for (; p + 1 < p1; p += 2) {  // two blocks in flight, same order as one at a time
        const int j0 = __ldg(ci + p), j1 = __ldg(ci + p + 1);
        T a0[B], a1[B], x0[B], x1[B];
        load_row<B>(lu + ((size_t)p * B + lane) * B, a0);
        load_row<B>(lu + ((size_t)(p + 1) * B + lane) * B, a1);
        load_row<B>(x + (size_t)j0 * B, x0);
        load_row<B>(x + (size_t)j1 * B, x1);
        acc = fnma_row<B>(a0, x0, acc);
        acc = fnma_row<B>(a1, x1, acc);
      }
      if (p < p1) {
        const int j0 = __ldg(ci + p);
        T a0[B], x0[B];
        load_row<B>(lu + ((size_t)p * B + lane) * B, a0);
        load_row<B>(x + (size_t)j0 * B, x0);
        acc = fnma_row<B>(a0, x0, acc);
      }
    }
    T out = T(0);
    const T* ui = uinv + ((size_t)(active ? i : 0) * B + (lane < B ? lane : 0)) * B;
#pragma unroll
    for (int c = 0; c < B; ++c) {
      T ac = __shfl_sync(0xffffffffu, acc, c, GP);
      if (active) out = fma(__ldg(ui + c), ac, out);
    }
    if (active) {
      x[(size_t)i * B + lane] = out;
      w[(size_t)i * B + lane] += out;
    }
  }
}

template <typename T>
__global__ void prolong_p_kernel(int b, int nb, const T* __restrict__ e, T* __restrict__ w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
    w[(size_t)i * b] += e[i];
}

// ----------------------------------------------------------------------------------
// scalar CSR level kernels: TPR lanes per row
// ----------------------------------------------------------------------------------

template <typename T, int TPR>
__global__ void __launch_bounds__(kThreads) csr_gs_colour_kernel(
    int r0, int r1, const int* __restrict__ rp, const int* __restrict__ ci,
    const T* __restrict__ v, const int* __restrict__ dpos, const T* __restrict__ rdiag,
    const T* __restrict__ b, T* __restrict__ x, bool lower_only,
    const unsigned char* __restrict__ rmask) {
  const int lane = threadIdx.x % TPR;
  const int rpb = blockDim.x / TPR;
  for (int base = r0 + blockIdx.x * rpb; base < r1; base += gridDim.x * rpb) {
    const int i = base + threadIdx.x / TPR;
    T s = T(0), bi = T(0), di = T(0);
    const bool live = (i < r1) && (!rmask || rmask[i]);
    if (live) {
      if (lane == 0) {  // issued with the row's first loads, not after the reduction
        bi = __ldg(b + i);
        di = __ldg(rdiag + i);
      }
      const int p0 = __ldg(rp + i), pd = __ldg(dpos + i);
      const int p1 = lower_only ? pd : __ldg(rp + i + 1);
      for (int p = p0 + lane; p < p1; p += TPR) {
        if (p == pd) continue;
        s = fma(__ldg(v + p), x[__ldg(ci + p)], s);
      }
    }
    s = group_sum<TPR>(s);
    if (live && lane == 0) x[i] = (bi - s) * di;
  }
}

// One colour of a PGS-MC sweep over the ELL copy of a level: TPR lanes per row, lane t
// owning slots t, t + TPR, ... of the row's K (row-major: slot k of row i at i*K + k).
// Every lane loads all its slots whatever the row's length (unused slots hold (i, 0)), so
// the only load that waits for another is the gather of x: two dependent trips to memory
// instead of three (row pointer, then entries, then x).  Rows longer than K (meta < 0)
// walk their CSR row instead.
// PDL: launched as a programmatic dependent of the previous kernel; the grid lets the next
// colour launch at once and loads what no kernel of the sweep writes (the slots, meta,
// 1/diagonal) before it waits for the previous colour, so only the gather of x and b
// remain after the dependency resolves.
template <typename T, int K, int TPR, bool PDL>
__global__ void __launch_bounds__(kThreads) ell_gs_colour_kernel(
    int r0, int r1, const int* __restrict__ ell_ci, const T* __restrict__ ell_v,
    const int* __restrict__ meta, const int* __restrict__ rp, const int* __restrict__ ci,
    const T* __restrict__ v, const int* __restrict__ dpos, const T* __restrict__ rdiag,
    const T* __restrict__ b, T* __restrict__ x, bool lower_only,
    const unsigned char* __restrict__ rmask) {
  constexpr int S = (K + TPR - 1) / TPR;  // slots per lane
  const int lane = threadIdx.x % TPR;
  const int rpb = blockDim.x / TPR;
  if constexpr (PDL) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int base = r0 + blockIdx.x * rpb; base < r1; base += gridDim.x * rpb) {
    const int i = base + threadIdx.x / TPR;
    T s = T(0), bi = T(0), di = T(0);
    const bool live = (i < r1) && (!rmask || rmask[i]);
    int m = 0;
    int j[S];
    T a[S], xj[S];
    if (live) {
      m = __ldg(meta + i);
      if (lane == 0) di = __ldg(rdiag + i);
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const int k = lane + q * TPR;
        j[q] = k < K ? __ldg(ell_ci + (size_t)i * K + k) : i;
        a[q] = k < K ? __ldg(ell_v + (size_t)i * K + k) : T(0);
      }
    }
    if constexpr (PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (live) {
      if (lane == 0) bi = b[i];
#pragma unroll
      for (int q = 0; q < S; ++q) xj[q] = x[j[q]];
      // lower_only: x of the later colours is stale, only the entries left of the diagonal
      const int used = lower_only ? (m >> 16) : K;
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (lane + q * TPR < used) s = fma(a[q], xj[q], s);
      if (m < 0) {
        const int p0 = __ldg(rp + i), pd = __ldg(dpos + i);
        const int p1 = lower_only ? pd : __ldg(rp + i + 1);
        for (int p = p0 + lane; p < p1; p += TPR) {
          if (p == pd) continue;
          s = fma(__ldg(v + p), x[__ldg(ci + p)], s);
        }
      }
    }
    s = group_sum<TPR>(s);
    if (live && lane == 0) x[i] = (bi - s) * di;
  }
}

// bc[I] = sum over the members i of aggregate I of (b_i - (A x)_i), over the ELL copy of
// the level: a group of 4*TPR lanes per aggregate takes four members at a time, TPR lanes
// per member and S slots per lane, so the member list, the entries and the gather of x
// are the only dependent trips to memory.  Rows longer than K (meta < 0) walk their CSR
// row (diagonal included) instead of the slots and the diagonal term.
template <typename T, int K, int TPR>
__global__ void __launch_bounds__(kThreads) ell_residual_restrict_kernel(
    int nc, const int* __restrict__ mptr, const int* __restrict__ members,
    const int* __restrict__ ell_ci, const T* __restrict__ ell_v, const int* __restrict__ meta,
    const T* __restrict__ diag, const int* __restrict__ rp, const int* __restrict__ ci,
    const T* __restrict__ v, const T* __restrict__ b, const T* __restrict__ x,
    T* __restrict__ bc, const unsigned char* __restrict__ cmask) {
  constexpr int kMembers = 4, G = kMembers * TPR, S = (K + TPR - 1) / TPR;
  const int lane = threadIdx.x % G;
  const int ms = lane / TPR, t = lane % TPR;
  const int gpb = blockDim.x / G;
  for (int base = blockIdx.x * gpb; base < nc; base += gridDim.x * gpb) {
    const int I = base + threadIdx.x / G;
    T total = T(0);
    // cmask: aggregates of the batched instances still iterating (the others keep stale
    // values that no active row reads)
    const bool live = I < nc && (!cmask || cmask[I]);
    if (live) {
      const int m0 = __ldg(mptr + I), m1 = __ldg(mptr + I + 1);
      for (int mb = m0 + ms; mb < m1; mb += kMembers) {
        const int i = __ldg(members + mb);
        const int m = __ldg(meta + i);
        if (t == 0) total += __ldg(b + i);
        int j[S];
        T a[S], xj[S];
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const int k = t + q * TPR;
          j[q] = k < K ? __ldg(ell_ci + (size_t)i * K + k) : i;
          a[q] = k < K ? __ldg(ell_v + (size_t)i * K + k) : T(0);
        }
        const T di = t == 0 ? __ldg(diag + i) : T(0);
        const T xi = t == 0 ? __ldg(x + i) : T(0);
#pragma unroll
        for (int q = 0; q < S; ++q) xj[q] = __ldg(x + j[q]);
        if (m >= 0) {
          total = fma(-di, xi, total);
#pragma unroll
          for (int q = 0; q < S; ++q) total = fma(-a[q], xj[q], total);
        } else {
          const int p1 = __ldg(rp + i + 1);
          for (int p = __ldg(rp + i) + t; p < p1; p += TPR)
            total = fma(-__ldg(v + p), __ldg(x + __ldg(ci + p)), total);
        }
      }
    }
    total = group_sum<G>(total);
    if (live && lane == 0) bc[I] = total;
  }
}

// The smoothers Section 5.1.1 compares PGS-MC with, in natural (storage) order.
// PJAC-NO: x_i = (b_i - sum_{j != i} a_ij x0_j) / a_ii for every row (x0: the values at
// the start of the sweep, a separate copy).
template <typename T>
__global__ void __launch_bounds__(kThreads) jacobi_sweep_kernel(
    int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
    const int* __restrict__ dpos, const T* __restrict__ rdiag, const T* __restrict__ b,
    const T* __restrict__ x0, T* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1), pd = __ldg(dpos + i);
    T s = T(0);
    for (int p = p0; p < p1; ++p)
      if (p != pd) s = fma(__ldg(v + p), __ldg(x0 + __ldg(ci + p)), s);
    x[i] = (__ldg(b + i) - s) * __ldg(rdiag + i);
  }
}

// PGS-NO: Gauss-Seidel through each chunk of kPgsNoChunk consecutive rows in order
// (forward) or reverse order (backward) with the chunk's new values; rows of other chunks
// are read at their values from the start of the sweep (x0).  One lane per row, two
// chunks per warp: every lane first sums its row's terms outside the chunk (all at
// once), then the chunk's rows take their turn one after another, each adding its
// terms inside the chunk (warp barrier between turns, so each sees the rows before it).
constexpr int kPgsNoChunk = 16;
template <typename T>
__global__ void __launch_bounds__(kThreads) pgs_no_sweep_kernel(
    int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
    const int* __restrict__ dpos, const T* __restrict__ rdiag, const T* __restrict__ b,
    const T* __restrict__ x0, T* x, bool forward) {
  static_assert(kWarp % kPgsNoChunk == 0, "whole chunks per warp");
  constexpr int kPerWarp = kWarp / kPgsNoChunk;
  const int nchunks = (n + kPgsNoChunk - 1) / kPgsNoChunk;
  const int t = threadIdx.x % kPgsNoChunk;
  const int warps = gridDim.x * (blockDim.x / kWarp);
  const int wid = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  // the loop bound depends on the warp only: every lane reaches the warp barriers
  for (int wbase = wid * kPerWarp; wbase < nchunks; wbase += warps * kPerWarp) {
    const int c = wbase + (threadIdx.x % kWarp) / kPgsNoChunk;
    const int c0 = c * kPgsNoChunk, c1 = min(c0 + kPgsNoChunk, n);
    const int i = c0 + t;
    const bool active = c < nchunks && i < c1;
    T off = T(0), bi = T(0), di = T(0);
    int p0 = 0, p1 = 0;
    if (active) {
      p0 = __ldg(rp + i);
      p1 = __ldg(rp + i + 1);
      bi = __ldg(b + i);
      di = __ldg(rdiag + i);
      for (int p = p0; p < p1; ++p) {
        const int j = __ldg(ci + p);
        if (j < c0 || j >= c1) off = fma(__ldg(v + p), __ldg(x0 + j), off);
      }
    }
    for (int turn = 0; turn < kPgsNoChunk; ++turn) {
      if (active && t == (forward ? turn : kPgsNoChunk - 1 - turn)) {
        T s = off;
        for (int p = p0; p < p1; ++p) {
          const int j = __ldg(ci + p);
          if (j >= c0 && j < c1 && j != i) s = fma(__ldg(v + p), x[j], s);
        }
        x[i] = (bi - s) * di;
      }
      __syncwarp();
    }
  }
}

// one group of TPR lanes per coarse row I; members of I processed in ascending order
template <typename T, int TPR>
__global__ void __launch_bounds__(kThreads) csr_residual_restrict_kernel(
    int nc, const int* __restrict__ mptr, const int* __restrict__ members,
    const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
    const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ bc,
    const unsigned char* __restrict__ cmask) {
  const int lane = threadIdx.x % TPR;
  const int rpb = blockDim.x / TPR;
  for (int base = blockIdx.x * rpb; base < nc; base += gridDim.x * rpb) {
    const int I = base + threadIdx.x / TPR;
    T total = T(0);
    const bool live = I < nc && (!cmask || cmask[I]);
    if (live) {
      const int m0 = __ldg(mptr + I), m1 = __ldg(mptr + I + 1);
      for (int m = m0; m < m1; ++m) {
        const int i = __ldg(members + m);
        T s = T(0);
        const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
        for (int p = p0 + lane; p < p1; p += TPR) s = fma(__ldg(v + p), __ldg(x + __ldg(ci + p)), s);
        total += (lane == 0 ? b[i] : T(0)) - s;
      }
    }
    total = group_sum<TPR>(total);
    if (live && lane == 0) bc[I] = total;
  }
}

template <typename T>
__global__ void prolong_add_kernel(int n, const int* __restrict__ agg, const T* __restrict__ xc,
                                   T* __restrict__ x, const unsigned char* __restrict__ fmask) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!fmask || fmask[i]) x[i] += xc[agg[i]];
}

// x = Ainv b: four warps per row (interleaved 32-column slices, four accumulators per
// lane), the warps' sums added in a fixed order through shared memory
constexpr int kGemvWarpsPerRow = 4;
template <typename T>
__global__ void __launch_bounds__(kThreads) dense_gemv_kernel(int n, const double* __restrict__ A,
                                                             const T* __restrict__ b,
                                                             T* __restrict__ x) {
  constexpr int kW = kGemvWarpsPerRow, kStep = kW * kWarp;
  constexpr int kRows = kThreads / kWarp / kW;  // rows per block
  __shared__ double part[kThreads / kWarp];
  const int lane = threadIdx.x % kWarp, wib = threadIdx.x / kWarp;
  const int sub = wib % kW;
  // the loop bound depends on the block only: every thread reaches both barriers
  for (int r0 = blockIdx.x * kRows; r0 < n; r0 += gridDim.x * kRows) {
    const int r = r0 + wib / kW;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (r < n) {
      const double* row = A + (size_t)r * n;
      int c = sub * kWarp + lane;
      for (; c + 3 * kStep < n; c += 4 * kStep) {
        s0 = fma(__ldg(row + c), (double)__ldg(b + c), s0);
        s1 = fma(__ldg(row + c + kStep), (double)__ldg(b + c + kStep), s1);
        s2 = fma(__ldg(row + c + 2 * kStep), (double)__ldg(b + c + 2 * kStep), s2);
        s3 = fma(__ldg(row + c + 3 * kStep), (double)__ldg(b + c + 3 * kStep), s3);
      }
      for (; c < n; c += kStep) s0 = fma(__ldg(row + c), (double)__ldg(b + c), s0);
    }
    const double s = group_sum<kWarp>((s0 + s1) + (s2 + s3));
    __syncthreads();  // the previous rows' reads of part are done
    if (lane == 0) part[wib] = s;
    __syncthreads();
    if (threadIdx.x < kRows && r0 + (int)threadIdx.x < n) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < kW; ++q) t += part[threadIdx.x * kW + q];
      x[r0 + threadIdx.x] = (T)t;
    }
  }
}

__global__ void cast_d2f_kernel(size_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void cast_f2d_kernel(size_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// ----------------------------------------------------------------------------------
// Krylov reductions (deterministic: per-block partials, then a fixed-order sum)
// ----------------------------------------------------------------------------------
constexpr int kDotChunk = 8;
constexpr int kMaxK = kKrylovMaxK;
constexpr int kMaxRestart = 64;  // msp_config.restart <= 64

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = group_sum<kWarp>(v);
  const int w = threadIdx.x / kWarp, l = threadIdx.x % kWarp;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < blockDim.x / kWarp) t = sh[threadIdx.x];
  if (w == 0) t = group_sum<kWarp>(t);
  return t;  // valid in thread 0
}

// 8 accumulators per lane summed over the warp by a transposing butterfly: at each level a
// lane keeps half of its values and receives the other half from its partner, 9 shuffles
// and 9 FP64 adds per lane in all (8 separate trees would take 40 adds, a sixth of the
// kernel's FP64 work at this size).  Lane l with l % 4 == 0 returns accumulator
// 4*bit4(l) + 2*bit3(l) + bit2(l).
__device__ __forceinline__ double transpose_sum8(double (&a)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double send = h16 ? a[q] : a[q + 4];
    const double keep = h16 ? a[q + 4] : a[q];
    a[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double send = h8 ? a[q] : a[q + 2];
    const double keep = h8 ? a[q + 2] : a[q];
    a[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double send = h4 ? a[0] : a[1];
  const double keep = h4 ? a[1] : a[0];
  double r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

__global__ void set_int_kernel(int* __restrict__ p, int v) { *p = v; }

// One right-hand vector, four elements in flight per thread: partial[b * stride + k] =
// V_k . x over block b's share, k < K.  With `jsel` (a device index j, read at run time) the
// kernel takes K = j + 1 and x = V_j, the basis against its newest vector, so that one
// captured launch serves every step; j < 0 makes it return at once.  The basis is read
// with evict-first loads: it is streamed once, and the kernel may run beside other work
// whose data should stay in L2.
__global__ void __launch_bounds__(kThreads) multi_dot1_kernel(size_t n, const double* __restrict__ V,
                                                             size_t ldv, int K,
                                                             const double* __restrict__ x,
                                                             double* __restrict__ partial,
                                                             int stride,
                                                             const int* __restrict__ jsel) {
  static_assert(kDotChunk == 8 && kThreads == 256, "the reduction below is for 8 x 8 warps");
  __shared__ double sh[kThreads / kWarp][kDotChunk];
  if (jsel) {
    const int j = *jsel;
    if (j < 0 || j + 1 > stride) return;  // uniform over the grid
    K = j + 1;
    x = V + (size_t)j * ldv;
  }
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  for (int k0 = 0; k0 < K; k0 += kDotChunk) {
    const int kc = min(kDotChunk, K - k0);
    double a[kDotChunk];
#pragma unroll
    for (int k = 0; k < kDotChunk; ++k) a[k] = 0.0;
    const size_t G = (size_t)gridDim.x * blockDim.x;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; i + 3 * G < n; i += 4 * G) {
      double u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) u[q] = x[i + q * G];
#pragma unroll
      for (int k = 0; k < kDotChunk; ++k)
        if (k < kc) {
          double vk[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) vk[q] = __ldcs(V + (size_t)(k0 + k) * ldv + i + q * G);
#pragma unroll
          for (int q = 0; q < 4; ++q) a[k] = fma(vk[q], u[q], a[k]);
        }
    }
    for (; i < n; i += G) {
      const double u = x[i];
#pragma unroll
      for (int k = 0; k < kDotChunk; ++k)
        if (k < kc) a[k] = fma(__ldcs(V + (size_t)(k0 + k) * ldv + i), u, a[k]);
    }
    const double r = transpose_sum8(a, lane);
    __syncthreads();  // the previous chunk's reads of sh are done
    if ((lane & 3) == 0) sh[wid][slot] = r;
    __syncthreads();
    if (threadIdx.x < kc) {  // fixed order over the warps
      double t = 0.0;
#pragma unroll
      for (int w2 = 0; w2 < kThreads / kWarp; ++w2) t += sh[w2][threadIdx.x];
      partial[(size_t)blockIdx.x * stride + k0 + threadIdx.x] = t;
    }
  }
}

// out[k] = sum over blocks of partial[b * stride + k], k < K (one warp per output, the
// warps of the grid striding over the outputs); with `jsel` (launched as one block),
// K = *jsel + 1 (nothing when *jsel < 0) and, once every thread has read it, the index
// moves on to the next step: *jsel = j + 1
__global__ void reduce_partials_strided_kernel(int K, int nblocks, int stride,
                                               const double* __restrict__ partial,
                                               double* __restrict__ out,
                                               int* __restrict__ jsel) {
  const int j = jsel ? *jsel : 0;
  if (jsel) K = j < 0 ? 0 : min(j + 1, stride);
  const int wpb = blockDim.x / kWarp, lane = threadIdx.x % kWarp;
  for (int k = blockIdx.x * wpb + threadIdx.x / kWarp; k < K; k += gridDim.x * wpb) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += kWarp) s += partial[(size_t)b * stride + k];
    s = group_sum<kWarp>(s);
    if (lane == 0) out[k] = s;
  }
  if (jsel) {
    __syncthreads();  // every thread has read *jsel
    if (threadIdx.x == 0 && j >= 0) *jsel = j + 1;
  }
}

// One-pass Gram-Schmidt of FGMRES step j (one warp, j < 64).  The
// stored basis U = [u_0 .. u_j] is orthogonalised once; the orthonormal basis it stands for
// is Q = U T^-1 with T upper triangular (column k of T holds c_k = Q_k^T u_k above the
// diagonal and nu_k = ||u_k - Q_k c_k|| on it), so Q is never formed.  Inputs: d[k] = u_k .
// u_j and d[K + k] = u_k . w for k < K = j + 2 (u_{j+1} stands for w).  Computes
//   c_j = T_j^-T d[0..j-1], nu_j^2 = d[j] - |c_j|^2           (column j of T)
//   h = T_{j+1}^-T d[K .. K+j]                                (h = Q^T w, Arnoldi column)
//   g = T_{j+1}^-1 h                                          (w - Q h = w - U g)
// out[0..j] = h, out[72 + k] = c_j[k], out[144] = nu_j, out[145] = nu_j^2, out[146] = w.w,
// out[147] = 1 if nu_j^2 <= 0 (u_j lies in span Q: the previous step broke down).
__device__ void dcgs_coef_body(int j, const double* __restrict__ d, double* __restrict__ T, int ldt,
                               double* __restrict__ g, double* __restrict__ out) {
  // One warp.  The triangle of T, the dot products and the reciprocal diagonal of T are
  // staged in shared memory; the three triangular solves are column-oriented: lane l owns
  // rows l and l + 32, and at step k the owner of row k finishes its unknown, which is
  // broadcast, and every lane removes that unknown's column from its rows — so a step costs
  // one shuffle and one FMA per lane on the critical path, not a row's dot product.  The
  // updates of a row come in the order of a row-by-row substitution (increasing column in
  // the two forward solves); the unknowns are the row's value times the stored reciprocal.
  constexpr int ld = kMaxRestart + 1;  // odd: the row reads of the forward solves are
                                       // spread over the banks
  __shared__ double sT[(kMaxRestart + 2) * ld];
  __shared__ double sd[2 * kMaxK], rd[kMaxRestart + 2];
  const int lane = threadIdx.x;
  const int K = j + 2;
  for (int q = lane; q < j * j; q += kWarp) {
    const int col = q / j, row = q % j;
    if (row <= col) sT[col * ld + row] = T[(size_t)col * ldt + row];
  }
  for (int q = lane; q < 2 * K; q += kWarp) sd[q] = d[q];
  for (int k = lane; k < j; k += kWarp) rd[k] = 1.0 / T[(size_t)k * ldt + k];
  __syncwarp();
  const int i0 = lane, i1 = lane + kWarp;  // the rows this lane owns
  // forward substitution with L = T^T (L[i][k] = T[k][i] = sT[i * ld + k]) over n rows of
  // the right-hand side rhs: returns the unknowns of rows i0 and i1
  auto forward = [&](int n, const double* rhs, double& x0, double& x1) {
    double r0 = i0 < n ? rhs[i0] : 0.0, r1 = i1 < n ? rhs[i1] : 0.0;
    x0 = 0.0;
    x1 = 0.0;
    for (int k = 0; k < n; ++k) {
      const bool hi = k >= kWarp;
      const double mine = (hi ? r1 : r0) * rd[k];
      const double xk = __shfl_sync(0xffffffffu, mine, k & (kWarp - 1));
      if (lane == (k & (kWarp - 1))) {
        if (hi) x1 = xk;
        else x0 = xk;
      }
      if (i0 > k && i0 < n) r0 = fma(-sT[i0 * ld + k], xk, r0);
      if (i1 > k && i1 < n) r1 = fma(-sT[i1 * ld + k], xk, r1);
    }
  };
  // c = T_j^-T (U_j^T u_j): column j of T above the diagonal
  double c0, c1;
  forward(j, sd, c0, c1);
  double c2 = (i0 < j ? c0 * c0 : 0.0) + (i1 < j ? c1 * c1 : 0.0);
#pragma unroll
  for (int o = kWarp / 2; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
  if (i0 < j) out[72 + i0] = c0;
  if (i1 < j) out[72 + i1] = c1;
  const double nu2 = sd[j] - c2;
  if (lane == 0) {
    out[145] = nu2;
    out[146] = sd[K + j + 1];
  }
  if (!(nu2 > 0.0)) {
    if (lane == 0) {
      out[144] = 0.0;
      out[147] = 1.0;
    }
    for (int k = lane; k <= j; k += kWarp) g[k] = 0.0;
    return;
  }
  const double nu = sqrt(nu2);
  // column j of T, stored by column
  if (i0 < j) {
    T[(size_t)j * ldt + i0] = c0;
    sT[j * ld + i0] = c0;
  }
  if (i1 < j) {
    T[(size_t)j * ldt + i1] = c1;
    sT[j * ld + i1] = c1;
  }
  if (lane == 0) {
    out[144] = nu;
    out[147] = 0.0;
    T[(size_t)j * ldt + j] = nu;
    sT[j * ld + j] = nu;
    rd[j] = 1.0 / nu;
  }
  __syncwarp();
  // h = T^-T (U^T w)
  double h0, h1;
  forward(j + 1, sd + K, h0, h1);
  if (i0 <= j) out[i0] = h0;
  if (i1 <= j) out[i1] = h1;
  // g = T^-1 h, back substitution by columns (column k of T: sT[k * ld + i], i <= k)
  double r0 = h0, r1 = h1, g0 = 0.0, g1 = 0.0;
  for (int k = j; k >= 0; --k) {
    const bool hi = k >= kWarp;
    const double mine = (hi ? r1 : r0) * rd[k];
    const double gk = __shfl_sync(0xffffffffu, mine, k & (kWarp - 1));
    if (lane == (k & (kWarp - 1))) {
      if (hi) g1 = gk;
      else g0 = gk;
    }
    if (i0 < k) r0 = fma(-sT[k * ld + i0], gk, r0);
    if (i1 < k) r1 = fma(-sT[k * ld + i1], gk, r1);
  }
  if (i0 <= j) g[i0] = g0;
  if (i1 <= j) g[i1] = g1;
}

__global__ void dcgs_coef_kernel(int j, const double* __restrict__ d, double* __restrict__ T,
                                 int ldt, double* __restrict__ g, double* __restrict__ out) {
  dcgs_coef_body(j, d, T, ldt, g, out);
}

// the same for every active instance of a batch (one block per instance; per-instance
// dot products, factor, coefficients and results at the given strides)
__global__ void dcgs_coef_batch_kernel(int j, const int* __restrict__ active,
                                       const double* __restrict__ d, int dstride,
                                       double* __restrict__ T, int tstride, int ldt,
                                       double* __restrict__ g, int gstride,
                                       double* __restrict__ out, int ostride) {
  const int i = blockIdx.x;
  if (!active[i]) return;  // uniform over the block
  dcgs_coef_body(j, d + (size_t)i * dstride, T + (size_t)i * tstride, ldt, g + (size_t)i * gstride,
                 out + (size_t)i * ostride);
}

// Column j + 1 of T from d[k] = u_k . u_{j+1}, k <= j + 1 (the last vector's own
// correction, computed when the Arnoldi column of step j must be final: at convergence, at
// MaxIt and at the end of a restart cycle).  out[72 + k] = c_{j+1}[k], out[144] = nu_{j+1},
// out[145] = nu_{j+1}^2, out[147] = 1 if nu_{j+1}^2 <= 0.
__device__ void dcgs_finalize_body(int j1, const double* __restrict__ d, double* __restrict__ T,
                                   int ldt, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double c2 = 0.0;
  for (int k = 0; k < j1; ++k) {
    double t = d[k];
    for (int i = 0; i < k; ++i) t -= T[(size_t)k * ldt + i] * out[72 + i];
    const double ck = t / T[(size_t)k * ldt + k];
    out[72 + k] = ck;
    c2 += ck * ck;
  }
  const double nu2 = d[j1] - c2;
  out[145] = nu2;
  const bool ok = nu2 > 0.0;
  out[144] = ok ? sqrt(nu2) : 0.0;
  out[147] = ok ? 0.0 : 1.0;
  if (ok) {
    for (int k = 0; k < j1; ++k) T[(size_t)j1 * ldt + k] = out[72 + k];
    T[(size_t)j1 * ldt + j1] = out[144];
  }
}

__global__ void dcgs_finalize_kernel(int j1, const double* __restrict__ d, double* __restrict__ T,
                                     int ldt, double* __restrict__ out) {
  dcgs_finalize_body(j1, d, T, ldt, out);
}

__global__ void dcgs_finalize_batch_kernel(int j1, const int* __restrict__ active,
                                           const double* __restrict__ d, int dstride,
                                           double* __restrict__ T, int tstride, int ldt,
                                           double* __restrict__ out, int ostride) {
  const int i = blockIdx.x;
  if (!active[i]) return;
  dcgs_finalize_body(j1, d + (size_t)i * dstride, T + (size_t)i * tstride, ldt,
                     out + (size_t)i * ostride);
}

// one warp per output k: lanes sum strided partials, then a fixed-order shuffle tree
__global__ void reduce_partials_kernel(int K, int nblocks, const double* __restrict__ partial,
                                       double* __restrict__ out, bool accumulate,
                                       const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int k = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const int lane = threadIdx.x % kWarp;
  if (k >= K) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += kWarp) s += partial[(size_t)b * kMaxK + k];
  s = group_sum<kWarp>(s);
  if (lane == 0) out[k] = accumulate ? out[k] + s : s;
}

__global__ void __launch_bounds__(kThreads) multi_axpy_norm_kernel(
    size_t n, const double* __restrict__ V, size_t ldv, int K, const double* __restrict__ h,
    double* __restrict__ w, double* __restrict__ partial, const int* __restrict__ gate) {
  __shared__ double sh[kThreads / kWarp];
  __shared__ double hs[kMaxK];
  if (gate && *gate == 0) return;
  for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  double nrm = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double wi = w[i];
    for (int k = 0; k < K; ++k) wi = fma(-hs[k], __ldg(V + (size_t)k * ldv + i), wi);
    w[i] = wi;
    nrm = fma(wi, wi, nrm);
  }
  double t = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxK] = t;
}

__global__ void __launch_bounds__(kThreads) norm2_partial_kernel(size_t n, const double* __restrict__ x,
                                                                double* __restrict__ partial) {
  __shared__ double sh[kThreads / kWarp];
  double nrm = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    nrm = fma(x[i], x[i], nrm);
  double t = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxK] = t;
}

// in place allowed (v == w); multiplies by the reciprocal (an FP64 division per element
// would make this kernel FP64-ALU bound)
__global__ void normalize_kernel(size_t n, const double* w, const double* __restrict__ nrm2,
                                 double* v, double* __restrict__ hn) {
  const double h = sqrt(nrm2[0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) hn[0] = h;
  if (h == 0.0) return;
  const double rh = 1.0 / h;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * rh;
}

// DGKS test after one Gram-Schmidt pass: gate = 1 iff ||w_after||^2 < ||w_before||^2 / 2

__global__ void update_x_kernel(size_t n, const double* __restrict__ Z, size_t ldz, int K,
                                const double* __restrict__ y, double* __restrict__ x) {
  __shared__ double ys[kMaxK];
  for (int k = threadIdx.x; k < K; k += blockDim.x) ys[k] = y[k];
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double xi = x[i];
    for (int k = 0; k < K; ++k) xi = fma(ys[k], __ldg(Z + (size_t)k * ldz + i), xi);
    x[i] = xi;
  }
}

__global__ void scale_kernel(size_t n, const double* __restrict__ r, double alpha,
                             double* __restrict__ v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] = r[i] * alpha;
}

// ---- batched Krylov: the vector of a block-diagonal system is split into chunks that each
// lie inside one instance (chunk c covers [cs[c], ce[c]) of instance ci[c]); every chunk
// writes its own partials and the partials of an instance are summed in chunk order, so
// the result is deterministic and does not depend on the other instances.  Chunks of an
// instance whose active[] flag is 0 are skipped.
__global__ void __launch_bounds__(kThreads) seg_multi_dot_kernel(
    int nchunks, const int* __restrict__ cs, const int* __restrict__ ce,
    const int* __restrict__ cinst, const int* __restrict__ active, const double* __restrict__ V,
    size_t ldv, int K, const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double sh[kThreads / kWarp][kDotChunk];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    if (!active[cinst[c]]) continue;  // uniform over the block
    const size_t i0 = cs[c], i1 = ce[c];
    for (int k0 = 0; k0 < K; k0 += kDotChunk) {
      const int kc = min(kDotChunk, K - k0);
      double acc[kDotChunk];
#pragma unroll
      for (int k = 0; k < kDotChunk; ++k) acc[k] = 0.0;
      for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < kDotChunk; ++k)
          if (k < kc) acc[k] = fma(__ldg(V + (size_t)(k0 + k) * ldv + i), wi, acc[k]);
      }
      const double r = transpose_sum8(acc, lane);
      __syncthreads();
      if ((lane & 3) == 0)
        sh[wid][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = r;
      __syncthreads();
      if (threadIdx.x < kc) {
        double t = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < kThreads / kWarp; ++w2) t += sh[w2][threadIdx.x];
        partial[(size_t)c * kMaxK + k0 + threadIdx.x] = t;
      }
    }
  }
}

// Two right-hand vectors per chunk: partial[c][k] = V_k . x0 and partial[c][K + k] = V_k .
// x1 over chunk c (row stride 2 * kMaxK), the chunks of the active instances only
__global__ void __launch_bounds__(kThreads) seg_multi_dot2_kernel(
    int nchunks, const int* __restrict__ cs, const int* __restrict__ ce,
    const int* __restrict__ cinst, const int* __restrict__ active, const double* __restrict__ V,
    size_t ldv, int K, const double* __restrict__ x0, const double* __restrict__ x1,
    double* __restrict__ partial) {
  __shared__ double sh[2][kThreads / kWarp][kDotChunk];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    if (!active[cinst[c]]) continue;  // uniform over the block
    const size_t i0 = cs[c], i1 = ce[c];
    for (int k0 = 0; k0 < K; k0 += kDotChunk) {
      const int kc = min(kDotChunk, K - k0);
      double a0[kDotChunk], a1[kDotChunk];
#pragma unroll
      for (int k = 0; k < kDotChunk; ++k) a0[k] = a1[k] = 0.0;
      for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double u = x0[i], w = x1[i];
#pragma unroll
        for (int k = 0; k < kDotChunk; ++k)
          if (k < kc) {
            const double vk = __ldg(V + (size_t)(k0 + k) * ldv + i);
            a0[k] = fma(vk, u, a0[k]);
            a1[k] = fma(vk, w, a1[k]);
          }
      }
      const double r0 = transpose_sum8(a0, lane);
      const double r1 = transpose_sum8(a1, lane);
      __syncthreads();
      if ((lane & 3) == 0) {
        sh[0][wid][slot] = r0;
        sh[1][wid][slot] = r1;
      }
      __syncthreads();
      if (threadIdx.x < 2 * kc) {
        const int r = threadIdx.x / kc, k = threadIdx.x % kc;
        double t = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < kThreads / kWarp; ++w2) t += sh[r][w2][k];
        partial[(size_t)c * (2 * kMaxK) + r * K + k0 + k] = t;
      }
    }
  }
}

// out[i * ostride + k] = sum over instance i's chunks (in order) of partial[c * pstride + k];
// one warp per (instance, k)
__global__ void seg_reduce_strided_kernel(int B, int K, const int* __restrict__ iptr,
                                          const int* __restrict__ ichunks,
                                          const int* __restrict__ active,
                                          const double* __restrict__ partial, int pstride,
                                          double* __restrict__ out, int ostride) {
  const int q = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const int lane = threadIdx.x % kWarp;
  if (q >= B * K) return;
  const int inst = q / K, k = q % K;
  if (!active[inst]) return;
  double s = 0.0;
  for (int t = iptr[inst] + lane; t < iptr[inst + 1]; t += kWarp)
    s += partial[(size_t)ichunks[t] * pstride + k];
  s = group_sum<kWarp>(s);
  if (lane == 0) out[(size_t)inst * ostride + k] = s;
}

// out[i * kMaxK + koff + k] = sum over instance i's chunks (in order) of partial[c][k];
// one warp per (instance, k)
__global__ void seg_reduce_kernel(int B, int K, const int* __restrict__ iptr,
                                  const int* __restrict__ ichunks, const int* __restrict__ active,
                                  const double* __restrict__ partial, double* __restrict__ out,
                                  int koff) {
  const int q = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const int lane = threadIdx.x % kWarp;
  if (q >= B * K) return;
  const int inst = q / K, k = q % K;
  if (!active[inst]) return;
  double s = 0.0;
  for (int t = iptr[inst] + lane; t < iptr[inst + 1]; t += kWarp)
    s += partial[(size_t)ichunks[t] * kMaxK + k];
  s = group_sum<kWarp>(s);
  if (lane == 0) out[(size_t)inst * kMaxK + koff + k] = s;
}

// w -= sum_k coef[inst][k] V[k] on every chunk of an active instance; partial[c][0] = sum of
// the new w^2 over the chunk
__global__ void __launch_bounds__(kThreads) seg_multi_axpy_norm_kernel(
    int nchunks, const int* __restrict__ cs, const int* __restrict__ ce,
    const int* __restrict__ cinst, const int* __restrict__ active, const double* __restrict__ V,
    size_t ldv, int K, const double* __restrict__ coef, double* __restrict__ w,
    double* __restrict__ partial) {
  __shared__ double sh[kThreads / kWarp];
  __shared__ double hs[kMaxK];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int inst = cinst[c];
    if (!active[inst]) continue;
    __syncthreads();  // the previous chunk's reads of hs are done
    for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = coef[(size_t)inst * kMaxK + k];
    __syncthreads();
    double nrm = 0.0;
    for (size_t i = cs[c] + threadIdx.x; i < (size_t)ce[c]; i += blockDim.x) {
      double wi = w[i];
      for (int k = 0; k < K; ++k) wi = fma(-hs[k], __ldg(V + (size_t)k * ldv + i), wi);
      w[i] = wi;
      nrm = fma(wi, wi, nrm);
    }
    const double t = block_sum(nrm, sh);
    if (threadIdx.x == 0) partial[(size_t)c * kMaxK] = t;
  }
}

// v = w / sqrt(nrm2[inst * kMaxK]) on the chunks of active instances (nothing where the
// norm is zero); in place allowed
__global__ void seg_normalize_kernel(int nchunks, const int* __restrict__ cs,
                                     const int* __restrict__ ce, const int* __restrict__ cinst,
                                     const int* __restrict__ active, const double* w,
                                     const double* __restrict__ nrm2, double* v) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int inst = cinst[c];
    if (!active[inst]) continue;
    const double h = sqrt(nrm2[(size_t)inst * kMaxK]);
    if (h == 0.0) continue;
    const double rh = 1.0 / h;
    for (size_t i = cs[c] + threadIdx.x; i < (size_t)ce[c]; i += blockDim.x) v[i] = w[i] * rh;
  }
}

// rmask[i] = active[row_inst[i]] != 0 for every level-0 row
__global__ void expand_mask_kernel(int nb, const int* __restrict__ row_inst,
                                   const int* __restrict__ active, unsigned char* __restrict__ rmask) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
    rmask[i] = active[row_inst[i]] != 0;
}

// v = 0 on the chunks of the instances with mask[inst] != 0
__global__ void seg_zero_kernel(int nchunks, const int* __restrict__ cs, const int* __restrict__ ce,
                                const int* __restrict__ cinst, const int* __restrict__ mask,
                                double* __restrict__ v) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    if (!mask[cinst[c]]) continue;
    for (size_t i = cs[c] + threadIdx.x; i < (size_t)ce[c]; i += blockDim.x) v[i] = 0.0;
  }
}

// x += sum_{k < count[inst]} y[inst][k] Z[k]
__global__ void seg_update_x_kernel(int nchunks, const int* __restrict__ cs,
                                    const int* __restrict__ ce, const int* __restrict__ cinst,
                                    const int* __restrict__ count, const double* __restrict__ Z,
                                    size_t ldz, const double* __restrict__ y,
                                    double* __restrict__ x) {
  __shared__ double ys[kMaxK];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int inst = cinst[c], K = count[inst];
    if (K <= 0) continue;
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) ys[k] = y[(size_t)inst * kMaxK + k];
    __syncthreads();
    for (size_t i = cs[c] + threadIdx.x; i < (size_t)ce[c]; i += blockDim.x) {
      double xi = x[i];
      for (int k = 0; k < K; ++k) xi = fma(ys[k], __ldg(Z + (size_t)k * ldz + i), xi);
      x[i] = xi;
    }
  }
}

__global__ void check_finite_kernel(size_t n, const double* __restrict__ x, int* flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) {
      atomicExch(flag, 1);
      return;
    }
}

__global__ void gather_blocks_kernel(int nb, int b, const int* __restrict__ perm,
                                     const double* __restrict__ in, double* __restrict__ out) {
  const size_t n = (size_t)nb * b;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t / b, r = t % b;
    out[t] = in[(size_t)perm[k] * b + r];
  }
}

__global__ void scatter_blocks_kernel(int nb, int b, const int* __restrict__ perm,
                                      const double* __restrict__ in, double* __restrict__ out) {
  const size_t n = (size_t)nb * b;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t / b, r = t % b;
    out[(size_t)perm[k] * b + r] = in[t];
  }
}

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

// grid covering `groups` thread groups of GP lanes, capped at 8 blocks per SM
inline unsigned grid_groups(size_t groups, int gp) {
  return grid_for(groups * (size_t)gp, kThreads, kRowGridPerSm);
}

}  // namespace

// a launch as a programmatic dependent of the previous kernel in the stream
template <typename... Args, typename... Act>
int launch_programmatic(void (*kern)(Args...), unsigned grid, cudaStream_t s, Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "cudaLaunchKernelEx", __FILE__, __LINE__);
    return MSP_ERR_CUDA;
  }
  return MSP_OK;
}

#define MSP_B_SWITCH(b, ...)  \
  switch (b) {                 \
    case 1: { constexpr int B_ = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int B_ = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int B_ = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int B_ = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int B_ = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int B_ = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int B_ = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int B_ = 8; __VA_ARGS__; } break; \
    default: return MSP_ERR_ARG; \
  }

template <typename T>
int launch_bsr_spmv(int b, int nb, const int* rp, const int* ci, const T* v, const T* x,
                    const T* g, T* y, bool residual, cudaStream_t s,
                    const unsigned char* rmask, LongRows lr) {
  if (nb <= 0) return MSP_OK;
  MSP_B_SWITCH(b, {
    const unsigned grid = with_long_rows(grid_groups(nb, Gp<B_>::v), lr.n);
    if (residual)
      bsr_spmv_kernel<B_, T, true><<<grid, kThreads, 0, s>>>(nb, rp, ci, v, x, g, y, rmask,
                                                             lr.rows, lr.n, lr.thr);
    else
      bsr_spmv_kernel<B_, T, false><<<grid, kThreads, 0, s>>>(nb, rp, ci, v, x, g, y, rmask,
                                                              lr.rows, lr.n, lr.thr);
  });
  return launch_status();
}

template <typename T>
int launch_bsr_restrict_p(int b, int nb, const int* rp, const int* ci, const T* v, const T* w,
                          const T* g, const T* omega, T* rP, T* r, cudaStream_t s,
                          const unsigned char* rmask, LongRows lr) {
  if (nb <= 0) return MSP_OK;
  MSP_B_SWITCH(b, {
    const unsigned grid = with_long_rows(grid_groups(nb, Gp<B_>::v), lr.n);
    if (r)
      bsr_restrict_p_kernel<B_, T, true><<<grid, kThreads, 0, s>>>(
          nb, rp, ci, v, w, g, omega, rP, r, rmask, lr.rows, lr.n, lr.thr);
    else
      bsr_restrict_p_kernel<B_, T, false><<<grid, kThreads, 0, s>>>(
          nb, rp, ci, v, w, g, omega, rP, r, rmask, lr.rows, lr.n, lr.thr);
  });
  return launch_status();
}

template <typename T>
int launch_bsr_col0_update(int b, int nb, const int* rp, const int* ci, const T* c0, const T* e,
                           T* r, T* w, cudaStream_t s, const unsigned char* rmask,
                           LongRows lr) {
  if (nb <= 0) return MSP_OK;
  MSP_B_SWITCH(b, {
    const unsigned grid = with_long_rows(grid_groups(nb, Gp<B_>::v), lr.n);
    bsr_col0_update_kernel<B_, T><<<grid, kThreads, 0, s>>>(nb, rp, ci, c0, e, r, w, rmask,
                                                            lr.rows, lr.n, lr.thr);
  });
  return launch_status();
}

template <typename T>
int launch_extract_col0(size_t nnzb, int b, const T* v, T* c0, cudaStream_t s) {
  if (!nnzb) return MSP_OK;
  extract_col0_kernel<T><<<grid_for(nnzb * b, kThreads), kThreads, 0, s>>>(nnzb, b, v, c0);
  return launch_status();
}

template <typename T>
int launch_bgs_colour(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                      const T* aN, const T* y, T* w, bool lower_only, bool zero_pressure,
                      cudaStream_t s, const unsigned char* rmask, LongRows lr) {
  if (r1 <= r0 || b < 2) return MSP_OK;
  if (lr.n > 0 && lr.n == r1 - r0) {  // a colour of long rows only (the well rows)
    switch (b) {
#define MSP_BGS_LONG_CASE(BB)                                                                  \
  case BB:                                                                                     \
    return launch_programmatic(bgs_long_colour_kernel<BB, T, true>, (unsigned)(r1 - r0), s, r0, \
                               rp, ci, dpos, aN, y, w, lower_only, zero_pressure, rmask);
      MSP_BGS_LONG_CASE(2)
      MSP_BGS_LONG_CASE(3)
      MSP_BGS_LONG_CASE(4)
      MSP_BGS_LONG_CASE(5)
      MSP_BGS_LONG_CASE(6)
      MSP_BGS_LONG_CASE(7)
      MSP_BGS_LONG_CASE(8)
#undef MSP_BGS_LONG_CASE
      default:
        return MSP_ERR_ARG;
    }
  }
  switch (b) {
#define MSP_BGS_CASE(BB)                                                                   \
  case BB: {                                                                               \
    const unsigned grid =                                                                  \
        with_long_rows(grid_for((size_t)(r1 - r0) * (BB - 1), kThreads, kRowGridPerSm), lr.n); \
    bgs_colour_kernel<BB, T><<<grid, kThreads, 0, s>>>(                                    \
        r0, r1, rp, ci, dpos, aN, y, w, lower_only, zero_pressure, rmask, lr.rows, lr.n,    \
        lr.thr);                                                                           \
  } break;
    MSP_BGS_CASE(2)
    MSP_BGS_CASE(3)
    MSP_BGS_CASE(4)
    MSP_BGS_CASE(5)
    MSP_BGS_CASE(6)
    MSP_BGS_CASE(7)
    MSP_BGS_CASE(8)
#undef MSP_BGS_CASE
    default:
      return MSP_ERR_ARG;
  }
  return launch_status();
}

template <typename T>
int launch_nscale(int b, int nb, const T* dNinv, const T* g, T* y, cudaStream_t s) {
  if (nb <= 0 || b < 2) return MSP_OK;
  const unsigned grid = grid_for((size_t)nb * (b - 1), kThreads);
  switch (b - 1) {
    case 1: nscale_kernel<1, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 2: nscale_kernel<2, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 3: nscale_kernel<3, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 4: nscale_kernel<4, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 5: nscale_kernel<5, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 6: nscale_kernel<6, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    case 7: nscale_kernel<7, T><<<grid, kThreads, 0, s>>>(nb, dNinv, g, y); break;
    default: return MSP_ERR_ARG;
  }
  return launch_status();
}

template <typename T>
int launch_bilu_fwd(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                    const T* lu, const T* r, T* y, cudaStream_t s, const unsigned char* rmask,
                    LongRows lr) {
  if (r1 <= r0) return MSP_OK;
  if (lr.n > 0 && lr.n == r1 - r0) {  // a colour of long rows only (the well rows)
    MSP_B_SWITCH(b, {
      MSP_TRY(launch_programmatic(bilu_fwd_long_colour_kernel<B_, T, true>, (unsigned)(r1 - r0),
                                  s, r0, rp, ci, dpos, lu, r, y, rmask));
    });
    return MSP_OK;
  }
  MSP_B_SWITCH(b, {
    const unsigned grid = with_long_rows(grid_groups(r1 - r0, Gp<B_>::v), lr.n);
    bilu_fwd_kernel<B_, T><<<grid, kThreads, 0, s>>>(r0, r1, rp, ci, dpos, lu, r, y, rmask,
                                                     lr.rows, lr.n, lr.thr);
  });
  return launch_status();
}

template <typename T>
int launch_bilu_bwd(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                    const T* lu, const T* uinv, const T* y, T* x, T* w, cudaStream_t s,
                    const unsigned char* rmask, LongRows lr) {
  if (r1 <= r0) return MSP_OK;
  if (lr.n > 0 && lr.n == r1 - r0) {  // a colour of long rows only (the well rows)
    MSP_B_SWITCH(b, {
      MSP_TRY(launch_programmatic(bilu_bwd_long_colour_kernel<B_, T, true>, (unsigned)(r1 - r0),
                                  s, r0, rp, ci, dpos, lu, uinv, y, x, w, rmask));
    });
    return MSP_OK;
  }
  MSP_B_SWITCH(b, {
    const unsigned grid = with_long_rows(grid_groups(r1 - r0, Gp<B_>::v), lr.n);
    bilu_bwd_kernel<B_, T><<<grid, kThreads, 0, s>>>(r0, r1, rp, ci, dpos, lu, uinv, y, x, w,
                                                     rmask, lr.rows, lr.n, lr.thr);
  });
  return launch_status();
}

template <typename T>
int launch_prolong_p(int b, int nb, const T* e, T* w, cudaStream_t s) {
  if (nb <= 0) return MSP_OK;
  prolong_p_kernel<T><<<grid_for(nb, kThreads), kThreads, 0, s>>>(b, nb, e, w);
  return launch_status();
}

// Lanes per row for the scalar CSR kernels, from the entries a row reads.  In FP64 the
// shuffle tree costs one FP64 add per lane and step, on a GPU whose FP64 rate is ~1/32 of
// its FP32 rate, so short rows take one thread each; FP32 rows favour coalesced lanes.
template <typename T>
int csr_lanes(int len) {
  if constexpr (sizeof(T) == 8)
    return len <= 8 ? 1 : len <= 16 ? 2 : len <= 48 ? 4 : 8;
  else
    return len <= 4 ? 4 : len <= 12 ? 8 : 16;
}

#define MSP_TPR_SWITCH(tpr, ...)          \
  switch (tpr) {                         \
    case 1: { constexpr int TPR_ = 1; __VA_ARGS__; } break;   \
    case 2: { constexpr int TPR_ = 2; __VA_ARGS__; } break;   \
    case 4: { constexpr int TPR_ = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int TPR_ = 8; __VA_ARGS__; } break;   \
    default: { constexpr int TPR_ = 16; __VA_ARGS__; } break; \
  }

template <typename T>
int launch_csr_gs_colour(int r0, int r1, const int* rp, const int* ci, const T* v,
                         const int* dpos, const T* rdiag, const T* b, T* x, bool lower_only,
                         int avg_row, cudaStream_t s, const unsigned char* rmask) {
  if (r1 <= r0) return MSP_OK;
  const int tpr = csr_lanes<T>(lower_only ? (avg_row + 1) / 2 : avg_row);
  MSP_TPR_SWITCH(tpr, csr_gs_colour_kernel<T, TPR_><<<grid_groups(r1 - r0, TPR_), kThreads, 0, s>>>(
                          r0, r1, rp, ci, v, dpos, rdiag, b, x, lower_only, rmask));
  return launch_status();
}


// lanes per row of the ELL kernels by default (measured: one lane per 4 slots, 8 at most)
int ell_default_tpr(int K) { return K <= 8 ? 2 : (K <= 16 ? 4 : 8); }

// the (K, TPR) pairs the ELL kernels are built for: at most 8 slots per lane
bool ell_tpr_ok(int K, int tpr) {
  if (tpr != 2 && tpr != 4 && tpr != 8) return false;
  if (K != 8 && K != 16 && K != 24 && K != 32) return false;
  return K / tpr <= 8 && tpr <= K;
}

template <typename T>
int launch_ell_gs_colour(int K, int r0, int r1, const int* ell_ci, const T* ell_v,
                         const int* meta, const int* rp, const int* ci, const T* v,
                         const int* dpos, const T* rdiag, const T* b, T* x, bool lower_only,
                         cudaStream_t s, const unsigned char* rmask, bool pdl, int tpr) {
  if (r1 <= r0) return MSP_OK;
  if (tpr == 0) tpr = ell_default_tpr(K);
  if (!ell_tpr_ok(K, tpr)) return MSP_ERR_ARG;
  const int key = K * 16 + tpr;
  switch (key) {
#define MSP_ELL_CASE(KK, TT)                                                                \
  case KK * 16 + TT:                                                                        \
    if (pdl) {                                                                              \
      MSP_TRY(launch_programmatic(ell_gs_colour_kernel<T, KK, TT, true>,                    \
                                  grid_groups(r1 - r0, TT), s, r0, r1, ell_ci, ell_v, meta, \
                                  rp, ci, v, dpos, rdiag, b, x, lower_only, rmask));        \
    } else {                                                                                \
      ell_gs_colour_kernel<T, KK, TT, false><<<grid_groups(r1 - r0, TT), kThreads, 0, s>>>( \
          r0, r1, ell_ci, ell_v, meta, rp, ci, v, dpos, rdiag, b, x, lower_only, rmask);   \
    }                                                                                       \
    break;
    MSP_ELL_CASE(8, 2)
    MSP_ELL_CASE(8, 4)
    MSP_ELL_CASE(8, 8)
    MSP_ELL_CASE(16, 2)
    MSP_ELL_CASE(16, 4)
    MSP_ELL_CASE(16, 8)
    MSP_ELL_CASE(24, 4)
    MSP_ELL_CASE(24, 8)
    MSP_ELL_CASE(32, 4)
    MSP_ELL_CASE(32, 8)
#undef MSP_ELL_CASE
    default:
      return MSP_ERR_ARG;
  }
  return launch_status();
}

template <typename T>
int launch_csr_residual_restrict(int nc, const int* mptr, const int* members, const int* rp,
                                 const int* ci, const T* v, const T* b, const T* x, T* bc,
                                 int avg_row, cudaStream_t s, const unsigned char* cmask) {
  if (nc <= 0) return MSP_OK;
  const int tpr = std::min(8, csr_lanes<T>(avg_row));
  MSP_TPR_SWITCH(tpr, csr_residual_restrict_kernel<T, TPR_><<<grid_groups(nc, TPR_), kThreads, 0, s>>>(
                          nc, mptr, members, rp, ci, v, b, x, bc, cmask));
  return launch_status();
}

template <typename T>
int launch_jacobi_sweep(int n, const int* rp, const int* ci, const T* v, const int* dpos,
                        const T* rdiag, const T* b, const T* x0, T* x, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  jacobi_sweep_kernel<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, dpos, rdiag,
                                                                      b, x0, x);
  return launch_status();
}

template <typename T>
int launch_pgs_no_sweep(int n, const int* rp, const int* ci, const T* v, const int* dpos,
                        const T* rdiag, const T* b, const T* x0, T* x, bool forward,
                        cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  const size_t lanes = (size_t)((n + kPgsNoChunk - 1) / kPgsNoChunk) * kPgsNoChunk;
  pgs_no_sweep_kernel<T><<<grid_for(lanes, kThreads), kThreads, 0, s>>>(n, rp, ci, v, dpos,
                                                                        rdiag, b, x0, x, forward);
  return launch_status();
}

template <typename T>
int launch_ell_residual_restrict(int K, int nc, const int* mptr, const int* members,
                                 const int* ell_ci, const T* ell_v, const int* meta,
                                 const T* diag, const int* rp, const int* ci, const T* v,
                                 const T* b, const T* x, T* bc, cudaStream_t s,
                                 const unsigned char* cmask, int tpr) {
  if (nc <= 0) return MSP_OK;
  if (tpr == 0) tpr = ell_default_tpr(K);
  if (!ell_tpr_ok(K, tpr)) return MSP_ERR_ARG;
  switch (K * 16 + tpr) {
#define MSP_ELLR_CASE(KK, TT)                                                               \
  case KK * 16 + TT:                                                                        \
    ell_residual_restrict_kernel<T, KK, TT><<<grid_groups(nc, 4 * TT), kThreads, 0, s>>>(   \
        nc, mptr, members, ell_ci, ell_v, meta, diag, rp, ci, v, b, x, bc, cmask);         \
    break;
    MSP_ELLR_CASE(8, 2)
    MSP_ELLR_CASE(8, 4)
    MSP_ELLR_CASE(8, 8)
    MSP_ELLR_CASE(16, 2)
    MSP_ELLR_CASE(16, 4)
    MSP_ELLR_CASE(16, 8)
    MSP_ELLR_CASE(24, 4)
    MSP_ELLR_CASE(24, 8)
    MSP_ELLR_CASE(32, 4)
    MSP_ELLR_CASE(32, 8)
#undef MSP_ELLR_CASE
    default:
      return MSP_ERR_ARG;
  }
  return launch_status();
}

template <typename T>
int launch_prolong_add(int n, const int* agg, const T* xc, T* x, cudaStream_t s,
                       const unsigned char* fmask) {
  if (n <= 0) return MSP_OK;
  prolong_add_kernel<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(n, agg, xc, x, fmask);
  return launch_status();
}

template <typename T>
int launch_dense_gemv(int n, const double* Ainv, const T* b, T* x, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  dense_gemv_kernel<T><<<grid_groups(n, kGemvWarpsPerRow * kWarp), kThreads, 0, s>>>(n, Ainv, b,
                                                                                    x);
  return launch_status();
}

int launch_cast_d2f(size_t n, const double* in, float* out, cudaStream_t s) {
  if (!n) return MSP_OK;
  cast_d2f_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, in, out);
  return launch_status();
}
int launch_cast_f2d(size_t n, const float* in, double* out, cudaStream_t s) {
  if (!n) return MSP_OK;
  cast_f2d_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, in, out);
  return launch_status();
}

int krylov_blocks() { return sm_count() * 4; }

int launch_reduce_partials_strided(int K, int nblocks, int stride, const double* partial,
                                   double* out, cudaStream_t s, int* jsel) {
  if (jsel) {  // one block: its threads all read the index before it moves on
    if (stride > kMaxK) return MSP_ERR_ARG;
    reduce_partials_strided_kernel<<<1, 32 * kWarp, 0, s>>>(0, nblocks, stride, partial, out,
                                                            jsel);
    return launch_status();
  }
  if (K <= 0) return MSP_OK;
  if (K > stride) return MSP_ERR_ARG;
  const int wpb = 4;
  reduce_partials_strided_kernel<<<(K + wpb - 1) / wpb, wpb * kWarp, 0, s>>>(K, nblocks, stride,
                                                                             partial, out, jsel);
  return launch_status();
}

int launch_set_int(int* p, int v, cudaStream_t s) {
  set_int_kernel<<<1, 1, 0, s>>>(p, v);
  return launch_status();
}

int launch_multi_dot1(size_t n, const double* V, size_t ldv, int K, const double* x,
                      double* partial, int stride, int nblocks, cudaStream_t s, const int* jsel) {
  if (stride > kMaxK || (!jsel && (K > stride || !x))) return MSP_ERR_ARG;
  if (!jsel && K <= 0) return MSP_OK;
  multi_dot1_kernel<<<nblocks, kThreads, 0, s>>>(n, V, ldv, K, x, partial, stride, jsel);
  return launch_status();
}

int launch_dcgs_coef(int j, const double* d, double* T, int ldt, double* g, double* out,
                     cudaStream_t s) {
  if (j < 0 || j >= kMaxRestart || j + 2 > kMaxK || j + 1 > ldt) return MSP_ERR_ARG;
  dcgs_coef_kernel<<<1, kWarp, 0, s>>>(j, d, T, ldt, g, out);
  return launch_status();
}

int launch_dcgs_finalize(int j1, const double* d, double* T, int ldt, double* out,
                         cudaStream_t s) {
  if (j1 < 1 || j1 + 1 > kMaxK || j1 + 1 > ldt) return MSP_ERR_ARG;
  dcgs_finalize_kernel<<<1, kWarp, 0, s>>>(j1, d, T, ldt, out);
  return launch_status();
}

int launch_reduce_partials(int K, int nblocks, const double* partial, double* out,
                           bool accumulate, cudaStream_t s, const int* gate) {
  if (K > kMaxK) return MSP_ERR_ARG;
  if (K <= 0) return MSP_OK;
  const int wpb = 4;  // warps (outputs) per block
  reduce_partials_kernel<<<(K + wpb - 1) / wpb, wpb * kWarp, 0, s>>>(K, nblocks, partial, out,
                                                                     accumulate, gate);
  return launch_status();
}

int launch_multi_axpy_norm(size_t n, const double* V, size_t ldv, int K, const double* h,
                           double* w, double* partial, int nblocks, cudaStream_t s,
                           const int* gate) {
  if (K > kMaxK) return MSP_ERR_ARG;
  multi_axpy_norm_kernel<<<nblocks, kThreads, 0, s>>>(n, V, ldv, K, h, w, partial, gate);
  return launch_status();
}

int launch_norm2_partial(size_t n, const double* x, double* partial, int nblocks,
                         cudaStream_t s) {
  norm2_partial_kernel<<<nblocks, kThreads, 0, s>>>(n, x, partial);
  return launch_status();
}

int launch_normalize(size_t n, const double* w, const double* nrm2, double* v, double* hn,
                     cudaStream_t s) {
  normalize_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, w, nrm2, v, hn);
  return launch_status();
}

int launch_update_x(size_t n, const double* Z, size_t ldz, int K, const double* y, double* x,
                    cudaStream_t s) {
  if (K > kMaxK) return MSP_ERR_ARG;
  if (K <= 0) return MSP_OK;
  update_x_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, Z, ldz, K, y, x);
  return launch_status();
}

int launch_scale(size_t n, const double* r, double alpha, double* v, cudaStream_t s) {
  scale_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, r, alpha, v);
  return launch_status();
}

int seg_grid(int nchunks) { return std::max(1, std::min(nchunks, krylov_blocks())); }

int launch_seg_multi_dot(const SegChunks& sc, const int* active, const double* V, size_t ldv,
                         int K, const double* w, double* partial, cudaStream_t s) {
  if (K > kMaxK) return MSP_ERR_ARG;
  if (K <= 0 || sc.n <= 0) return MSP_OK;
  seg_multi_dot_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(sc.n, sc.start, sc.end, sc.inst,
                                                           active, V, ldv, K, w, partial);
  return launch_status();
}

int launch_seg_reduce(const SegChunks& sc, int B, int K, const int* active,
                      const double* partial, double* out, int koff, cudaStream_t s) {
  if (K + koff > kMaxK) return MSP_ERR_ARG;
  if (K <= 0 || B <= 0) return MSP_OK;
  const int wpb = 4;
  const long long q = (long long)B * K;
  seg_reduce_kernel<<<(unsigned)((q + wpb - 1) / wpb), wpb * kWarp, 0, s>>>(
      B, K, sc.iptr, sc.ichunks, active, partial, out, koff);
  return launch_status();
}

int launch_seg_multi_dot2(const SegChunks& sc, const int* active, const double* V, size_t ldv,
                          int K, const double* x0, const double* x1, double* partial,
                          cudaStream_t s) {
  if (K > kMaxK) return MSP_ERR_ARG;
  if (K <= 0 || sc.n <= 0) return MSP_OK;
  seg_multi_dot2_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(sc.n, sc.start, sc.end, sc.inst,
                                                            active, V, ldv, K, x0, x1, partial);
  return launch_status();
}

int launch_seg_reduce_strided(const SegChunks& sc, int B, int K, const int* active,
                              const double* partial, int pstride, double* out, int ostride,
                              cudaStream_t s) {
  if (K > pstride || K > ostride) return MSP_ERR_ARG;
  if (K <= 0 || B <= 0) return MSP_OK;
  const int wpb = 4;
  const long long q = (long long)B * K;
  seg_reduce_strided_kernel<<<(unsigned)((q + wpb - 1) / wpb), wpb * kWarp, 0, s>>>(
      B, K, sc.iptr, sc.ichunks, active, partial, pstride, out, ostride);
  return launch_status();
}

int launch_dcgs_coef_batch(int B, int j, const int* active, const double* d, int dstride,
                           double* T, int tstride, int ldt, double* g, int gstride, double* out,
                           int ostride, cudaStream_t s) {
  if (B <= 0) return MSP_OK;
  if (j < 0 || j >= kMaxRestart || j + 2 > kMaxK || j + 1 > ldt) return MSP_ERR_ARG;
  dcgs_coef_batch_kernel<<<B, kWarp, 0, s>>>(j, active, d, dstride, T, tstride, ldt, g, gstride,
                                             out, ostride);
  return launch_status();
}

int launch_dcgs_finalize_batch(int B, int j1, const int* active, const double* d, int dstride,
                               double* T, int tstride, int ldt, double* out, int ostride,
                               cudaStream_t s) {
  if (B <= 0) return MSP_OK;
  if (j1 < 1 || j1 + 1 > kMaxK || j1 + 1 > ldt) return MSP_ERR_ARG;
  dcgs_finalize_batch_kernel<<<B, kWarp, 0, s>>>(j1, active, d, dstride, T, tstride, ldt, out,
                                                 ostride);
  return launch_status();
}

int launch_seg_multi_axpy_norm(const SegChunks& sc, const int* active, const double* V,
                               size_t ldv, int K, const double* coef, double* w, double* partial,
                               cudaStream_t s) {
  if (K > kMaxK) return MSP_ERR_ARG;
  if (sc.n <= 0) return MSP_OK;
  seg_multi_axpy_norm_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(
      sc.n, sc.start, sc.end, sc.inst, active, V, ldv, K, coef, w, partial);
  return launch_status();
}

int launch_seg_normalize(const SegChunks& sc, const int* active, const double* w,
                         const double* nrm2, double* v, cudaStream_t s) {
  if (sc.n <= 0) return MSP_OK;
  seg_normalize_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(sc.n, sc.start, sc.end, sc.inst,
                                                           active, w, nrm2, v);
  return launch_status();
}

int launch_expand_mask(int nb, const int* row_inst, const int* active, unsigned char* rmask,
                       cudaStream_t s) {
  if (nb <= 0) return MSP_OK;
  expand_mask_kernel<<<grid_for(nb, kThreads), kThreads, 0, s>>>(nb, row_inst, active, rmask);
  return launch_status();
}

int launch_seg_zero(const SegChunks& sc, const int* mask, double* v, cudaStream_t s) {
  if (sc.n <= 0) return MSP_OK;
  seg_zero_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(sc.n, sc.start, sc.end, sc.inst, mask, v);
  return launch_status();
}

int launch_seg_update_x(const SegChunks& sc, const int* count, const double* Z, size_t ldz,
                        const double* y, double* x, cudaStream_t s) {
  if (sc.n <= 0) return MSP_OK;
  seg_update_x_kernel<<<seg_grid(sc.n), kThreads, 0, s>>>(sc.n, sc.start, sc.end, sc.inst,
                                                          count, Z, ldz, y, x);
  return launch_status();
}

int launch_check_finite(size_t n, const double* x, int* flag, cudaStream_t s) {
  if (!n) return MSP_OK;
  check_finite_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, x, flag);
  return launch_status();
}

int launch_gather_blocks(int nb, int b, const int* perm, const double* in, double* out,
                         cudaStream_t s) {
  gather_blocks_kernel<<<grid_for((size_t)nb * b, kThreads), kThreads, 0, s>>>(nb, b, perm,
                                                                               in, out);
  return launch_status();
}

int launch_scatter_blocks(int nb, int b, const int* perm, const double* in, double* out,
                          cudaStream_t s) {
  scatter_blocks_kernel<<<grid_for((size_t)nb * b, kThreads), kThreads, 0, s>>>(nb, b, perm,
                                                                                in, out);
  return launch_status();
}

// explicit instantiations for the two value types of the preconditioner
#define MSP_INST(T)                                                                         \
  template int launch_bsr_spmv<T>(int, int, const int*, const int*, const T*, const T*,     \
                                  const T*, T*, bool, cudaStream_t, const unsigned char*,   \
                                  LongRows);                                                \
  template int launch_bsr_restrict_p<T>(int, int, const int*, const int*, const T*,         \
                                        const T*, const T*, const T*, T*, T*, cudaStream_t, \
                                        const unsigned char*, LongRows);                    \
  template int launch_bsr_col0_update<T>(int, int, const int*, const int*, const T*,        \
                                         const T*, T*, T*, cudaStream_t, const unsigned char*, \
                                         LongRows);                                          \
  template int launch_extract_col0<T>(size_t, int, const T*, T*, cudaStream_t);             \
  template int launch_bgs_colour<T>(int, int, int, const int*, const int*, const int*,      \
                                    const T*, const T*, T*, bool, bool, cudaStream_t,       \
                                    const unsigned char*, LongRows);                        \
  template int launch_nscale<T>(int, int, const T*, const T*, T*, cudaStream_t);            \
  template int launch_bilu_fwd<T>(int, int, int, const int*, const int*, const int*,        \
                                  const T*, const T*, T*, cudaStream_t, const unsigned char*, \
                                  LongRows);                                                \
  template int launch_bilu_bwd<T>(int, int, int, const int*, const int*, const int*,        \
                                  const T*, const T*, const T*, T*, T*, cudaStream_t,       \
                                  const unsigned char*, LongRows);                          \
  template int launch_prolong_p<T>(int, int, const T*, T*, cudaStream_t);                   \
  template int launch_csr_gs_colour<T>(int, int, const int*, const int*, const T*,          \
                                       const int*, const T*, const T*, T*, bool, int,       \
                                       cudaStream_t, const unsigned char*);                 \
  template int launch_ell_gs_colour<T>(int, int, int, const int*, const T*, const int*,      \
                                       const int*, const int*, const T*, const int*,      \
                                       const T*, const T*, T*, bool, cudaStream_t,        \
                                       const unsigned char*, bool, int);                  \
  template int launch_ell_residual_restrict<T>(int, int, const int*, const int*, const int*, \
                                               const T*, const int*, const T*, const int*,  \
                                               const int*, const T*, const T*, const T*, T*, \
                                               cudaStream_t, const unsigned char*, int);                               \
  template int launch_jacobi_sweep<T>(int, const int*, const int*, const T*, const int*,    \
                                      const T*, const T*, const T*, T*, cudaStream_t);      \
  template int launch_pgs_no_sweep<T>(int, const int*, const int*, const T*, const int*,    \
                                      const T*, const T*, const T*, T*, bool, cudaStream_t); \
  template int launch_csr_residual_restrict<T>(int, const int*, const int*, const int*,     \
                                               const int*, const T*, const T*, const T*,    \
                                               T*, int, cudaStream_t, const unsigned char*);                       \
  template int launch_prolong_add<T>(int, const int*, const T*, T*, cudaStream_t,             \
                                     const unsigned char*);          \
  template int launch_dense_gemv<T>(int, const double*, const T*, T*, cudaStream_t);
MSP_INST(double)
MSP_INST(float)
#undef MSP_INST

}  // namespace msp
