// Launchers of the CUDA kernels (host-callable).  All take a cudaStream_t and enqueue
// asynchronously; they return MSP_OK or MSP_ERR_CUDA (launch failure).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace msp {

// ---------------- solve phase: block rows of the colour-ordered BSR matrix --------------
// rmask (optional, one byte per row of the level-0 order): rows with rmask[i] == 0 are
// skipped — not read, not written (instances of a batch that have left the active set).
//
// Long rows (a well row couples to every perforated cell: ~nz blocks against <= 8 for a
// cell) would make one lane group walk a long dependent chain of loads while the rest of
// the launch waits for it.  Rows with more than `thr` blocks are taken by one thread
// block each, the row's blocks dealt round-robin over its threads and the partial sums
// combined in a fixed order (deterministic); `rows` lists exactly the rows of the
// launch's range with more than `thr` blocks, ascending.  The default (no list, thr =
// INT_MAX) leaves every row to its lane group.
struct LongRows {
  const int* rows = nullptr;
  int n = 0;
  int thr = 0x7fffffff;
};
// y = A x (residual = false) or y = g - A x (residual = true); b = block size 1..8.
template <typename T>
int launch_bsr_spmv(int b, int nb, const int* rp, const int* ci, const T* v, const T* x,
                    const T* g, T* y, bool residual, cudaStream_t s,
                    const unsigned char* rmask = nullptr, LongRows lr = LongRows());
// rP[i] = omega_i^T (g_i - (A w)_i)   (omega == nullptr: first unknown only); r != nullptr
// also receives g - A w
template <typename T>
int launch_bsr_restrict_p(int b, int nb, const int* rp, const int* ci, const T* v,
                          const T* w, const T* g, const T* omega, T* rP, T* r, cudaStream_t s,
                          const unsigned char* rmask = nullptr, LongRows lr = LongRows());
// r_i <- r_i - sum_j A_ij[:, 0] e_j and w_i[0] += e_i (r, w: nb*b values; c0: column 0 of
// every block, nnzb*b values; e: one value per block row)
template <typename T>
int launch_bsr_col0_update(int b, int nb, const int* rp, const int* ci, const T* c0, const T* e,
                           T* r, T* w, cudaStream_t s, const unsigned char* rmask = nullptr,
                           LongRows lr = LongRows());
// c0[p*b + r] = v[(p*b + r)*b]
template <typename T>
int launch_extract_col0(size_t nnzb, int b, const T* v, T* c0, cudaStream_t s);
// stage N: one block-GS sweep over the rows [r0, r1) of one colour on the (b-1)x(b-1)
// sub-blocks aN, pre-scaled by their row's D_N,i^-1, from y = D_N^-1 g (launch_nscale);
// reads/writes the concentration slots of w (stride b); lower_only for the first sweep
// from zero (later colours still hold zero).
template <typename T>
int launch_bgs_colour(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                      const T* aN, const T* y, T* w, bool lower_only, bool zero_pressure,
                      cudaStream_t s, const unsigned char* rmask = nullptr,
                      LongRows lr = LongRows());
// y[i*(b-1) + r] = (D_N,i^-1 g_i)[r] over the concentration unknowns of every block row
template <typename T>
int launch_nscale(int b, int nb, const T* dNinv, const T* g, T* y, cudaStream_t s);
// stage R: forward y_i = r_i - sum_{j<i} L_ij y_j and backward x_i = U_ii^-1 (y_i -
// sum_{j>i} U_ij x_j); the backward sweep also adds x_i into w.
template <typename T>
int launch_bilu_fwd(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                    const T* lu, const T* r, T* y, cudaStream_t s,
                    const unsigned char* rmask = nullptr, LongRows lr = LongRows());
template <typename T>
int launch_bilu_bwd(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                    const T* lu, const T* uinv, const T* y, T* x, T* w, cudaStream_t s,
                    const unsigned char* rmask = nullptr, LongRows lr = LongRows());
// w[i*b] += e[i]
template <typename T>
int launch_prolong_p(int b, int nb, const T* e, T* w, cudaStream_t s);

// ---------------- solve phase: scalar CSR AMG levels ----------------
// PGS-MC on rows [r0, r1) of one colour: x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii;
// lower_only: entries right of the diagonal are skipped (x there is still zero);
// avg_row: mean stored entries per row of the level (chooses the lanes per row).
template <typename T>
int launch_csr_gs_colour(int r0, int r1, const int* rp, const int* ci, const T* v,
                         const int* dpos, const T* rdiag, const T* b, T* x, bool lower_only,
                         int avg_row, cudaStream_t s, const unsigned char* rmask = nullptr);
// bc[I] = sum over members i of aggregate I (ascending) of (b_i - (A x)_i)
// the same sweep over the ELL copy of the level (K in {8, 16, 24, 32} slots per row, slot
// k of row i at i*K + k; meta from launch_build_ell; rows with meta < 0 use rp/ci/v);
// pdl: launched as a programmatic dependent of the previous kernel (constant operands are
// loaded before it waits for that kernel); tpr: lanes per row (2, 4 or 8 with at most 8
// slots per lane; 0: the default for K, ell_default_tpr)
template <typename T>
int launch_ell_gs_colour(int K, int r0, int r1, const int* ell_ci, const T* ell_v,
                         const int* meta, const int* rp, const int* ci, const T* v,
                         const int* dpos, const T* rdiag, const T* b, T* x, bool lower_only,
                         cudaStream_t s, const unsigned char* rmask = nullptr, bool pdl = false,
                         int tpr = 0);
// the same restriction over the ELL copy of the level (diag: a_ii of every row)
template <typename T>
int launch_ell_residual_restrict(int K, int nc, const int* mptr, const int* members,
                                 const int* ell_ci, const T* ell_v, const int* meta,
                                 const T* diag, const int* rp, const int* ci, const T* v,
                                 const T* b, const T* x, T* bc, cudaStream_t s,
                                 const unsigned char* cmask = nullptr, int tpr = 0);
int ell_default_tpr(int K);
bool ell_tpr_ok(int K, int tpr);
// PJAC-NO and PGS-NO sweeps in storage order (x0: the values at the start of the sweep,
// a separate copy; PGS-NO sweeps chunks of 16 consecutive rows)
template <typename T>
int launch_jacobi_sweep(int n, const int* rp, const int* ci, const T* v, const int* dpos,
                        const T* rdiag, const T* b, const T* x0, T* x, cudaStream_t s);
template <typename T>
int launch_pgs_no_sweep(int n, const int* rp, const int* ci, const T* v, const int* dpos,
                        const T* rdiag, const T* b, const T* x0, T* x, bool forward,
                        cudaStream_t s);
template <typename T>
int launch_csr_residual_restrict(int nc, const int* mptr, const int* members, const int* rp,
                                 const int* ci, const T* v, const T* b, const T* x, T* bc,
                                 int avg_row, cudaStream_t s, const unsigned char* cmask = nullptr);
// x_i += xc[agg[i]] (fmask: only the rows with fmask[i] != 0)
template <typename T>
int launch_prolong_add(int n, const int* agg, const T* xc, T* x, cudaStream_t s,
                       const unsigned char* fmask = nullptr);
// x = Ainv b (dense row-major n x n, FP64); b, x in the level's value type
template <typename T>
int launch_dense_gemv(int n, const double* Ainv, const T* b, T* x, cudaStream_t s);

// ---------------- precision casts ----------------
int launch_cast_d2f(size_t n, const double* in, float* out, cudaStream_t s);
int launch_cast_f2d(size_t n, const float* in, double* out, cudaStream_t s);

// ---------------- Krylov (FP64) ----------------
// one-pass Gram-Schmidt of FGMRES: dots of V[0..K) with one vector, strided reductions, and
// the small triangular solves of one step (kernel comments in solve_kernels.cu)
// out[k] = sum_b partial[b * stride + k], k < K; with jsel (device index j, K ignored):
// k <= j, then *jsel = j + 1 (unchanged when j < 0)
int launch_reduce_partials_strided(int K, int nblocks, int stride, const double* partial,
                                   double* out, cudaStream_t s, int* jsel = nullptr);
// *p = v in stream order (a kernel, so that it never waits behind host copies)
int launch_set_int(int* p, int v, cudaStream_t s);
// partial[b * stride + k] = block b's share of V_k . x, k < K; with jsel (device index j),
// K = j + 1 and x = V_j at run time (nothing when j < 0); stride <= kKrylovMaxK
int launch_multi_dot1(size_t n, const double* V, size_t ldv, int K, const double* x,
                      double* partial, int stride, int nblocks, cudaStream_t s,
                      const int* jsel = nullptr);
int launch_dcgs_coef(int j, const double* d, double* T, int ldt, double* g, double* out,
                     cudaStream_t s);
int launch_dcgs_finalize(int j1, const double* d, double* T, int ldt, double* out,
                         cudaStream_t s);
// out[k] = sum_b partial[b * kmax + k] (fixed order), k < K;  accumulate: out[k] += ...
int launch_reduce_partials(int K, int nblocks, const double* partial, double* out,
                           bool accumulate, cudaStream_t s, const int* gate = nullptr);
// w -= sum_k h[k] V[k]; partial[blk] = sum of w_new^2 over the block
int launch_multi_axpy_norm(size_t n, const double* V, size_t ldv, int K, const double* h,
                           double* w, double* partial, int nblocks, cudaStream_t s,
                           const int* gate = nullptr);
// v = w / sqrt(nrm2[0]) (nothing when the norm is zero); hn[0] = sqrt(nrm2[0])
int launch_normalize(size_t n, const double* w, const double* nrm2, double* v, double* hn,
                     cudaStream_t s);
// x += sum_k y[k] Z[k]
int launch_update_x(size_t n, const double* Z, size_t ldz, int K, const double* y, double* x,
                    cudaStream_t s);
// v = r / beta (beta a host scalar)
int launch_scale(size_t n, const double* r, double alpha, double* v, cudaStream_t s);
// partial[blk] = sum of x^2 over the block
int launch_norm2_partial(size_t n, const double* x, double* partial, int nblocks,
                         cudaStream_t s);
// nonfinite check: flag[0] = 1 if any entry is not finite
int launch_check_finite(size_t n, const double* x, int* flag, cudaStream_t s);
// out[k*b + r] = in[perm[k]*b + r]  (gather, b-blocks)
int launch_gather_blocks(int nb, int b, const int* perm, const double* in, double* out,
                         cudaStream_t s);
// out[perm[k]*b + r] = in[k*b + r]  (scatter, b-blocks)
int launch_scatter_blocks(int nb, int b, const int* perm, const double* in, double* out,
                          cudaStream_t s);

int krylov_blocks();  // number of blocks the reduction kernels use

// ---------------- batched Krylov over a block-diagonal system ----------------
// Chunks of the (colour-ordered) vector, each inside one instance: chunk c covers the
// elements [start[c], end[c]) of instance inst[c]; the chunks of instance i are
// ichunks[iptr[i] .. iptr[i+1]) in increasing order.  Partials: kmax per chunk.
struct SegChunks {
  int n = 0;
  const int* start = nullptr;
  const int* end = nullptr;
  const int* inst = nullptr;
  const int* iptr = nullptr;
  const int* ichunks = nullptr;
};
constexpr int kKrylovMaxK = 72;  // partial / coefficient stride per chunk and per instance
// partial[c][k] = V[k] . w over chunk c (active instances only)
int launch_seg_multi_dot(const SegChunks& sc, const int* active, const double* V, size_t ldv,
                         int K, const double* w, double* partial, cudaStream_t s);
// out[i][koff + k] = sum over instance i's chunks of partial[c][k] (active instances)
int launch_seg_reduce(const SegChunks& sc, int B, int K, const int* active,
                      const double* partial, double* out, int koff, cudaStream_t s);
// one-pass Gram-Schmidt of the batched solve: partial[c][k] = V[k] . x0 and
// partial[c][K + k] = V[k] . x1 over chunk c (stride 2 * kKrylovMaxK); a reduction with
// explicit strides; the per-instance triangular solves of a step (one block per instance)
int launch_seg_multi_dot2(const SegChunks& sc, const int* active, const double* V, size_t ldv,
                          int K, const double* x0, const double* x1, double* partial,
                          cudaStream_t s);
int launch_seg_reduce_strided(const SegChunks& sc, int B, int K, const int* active,
                              const double* partial, int pstride, double* out, int ostride,
                              cudaStream_t s);
int launch_dcgs_coef_batch(int B, int j, const int* active, const double* d, int dstride,
                           double* T, int tstride, int ldt, double* g, int gstride, double* out,
                           int ostride, cudaStream_t s);
int launch_dcgs_finalize_batch(int B, int j1, const int* active, const double* d, int dstride,
                               double* T, int tstride, int ldt, double* out, int ostride,
                               cudaStream_t s);
// w -= sum_k coef[i][k] V[k]; partial[c][0] = sum of the new w^2 over chunk c
int launch_seg_multi_axpy_norm(const SegChunks& sc, const int* active, const double* V,
                               size_t ldv, int K, const double* coef, double* w, double* partial,
                               cudaStream_t s);
// v = w / sqrt(nrm2[i][0]) per instance (nothing where the norm is zero)
int launch_seg_normalize(const SegChunks& sc, const int* active, const double* w,
                         const double* nrm2, double* v, cudaStream_t s);
// rmask[i] = (active[row_inst[i]] != 0) for the nb level-0 rows
int launch_expand_mask(int nb, const int* row_inst, const int* active, unsigned char* rmask,
                       cudaStream_t s);
// v = 0 on the instances with mask[i] != 0
int launch_seg_zero(const SegChunks& sc, const int* mask, double* v, cudaStream_t s);
// x += sum_{k < count[i]} y[i][k] Z[k]
int launch_seg_update_x(const SegChunks& sc, const int* count, const double* Z, size_t ldz,
                        const double* y, double* x, cudaStream_t s);

}  // namespace msp
