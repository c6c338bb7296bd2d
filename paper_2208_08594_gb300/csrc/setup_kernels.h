// Launchers of the setup kernels (host-callable, asynchronous on the given stream).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace msp {

// ---- bit-exact kernels (setup_exact.cu, compiled without FMA contraction) ----
// Inverse of every diagonal block (Gauss-Jordan, partial pivoting) and the quasi-IMPES
// weights omega_i = first row of D_i^-1.  flags->code = MSP_ERR_SINGULAR_BLOCK on a zero
// pivot (flags->index = block row).
int launch_diag_inverse(int b, int nb, const int* dpos, const double* v, double* dinv,
                        double* omega, DevFlags* flags, cudaStream_t s);
// Inverses of the (b-1)x(b-1) concentration sub-blocks of the diagonal blocks.
int launch_diagN_inverse(int b, int nb, const int* dpos, const double* v, double* dNinv,
                         DevFlags* flags, cudaStream_t s);
// A_P[p] = sum_k omega_i[k] * A_p[k][0] (decoupling) or A_p[0][0]
int launch_pressure_matrix(int b, int nb, const int* rp, const double* v, const double* omega,
                           bool decoupling, double* ap, cudaStream_t s);
// strength s_q = -(a_ij + a_ji)/2 on the adjacency entries q = (i, j) and the candidate
// flags s_q >= beta * max_k s_ik (max > 0)
int launch_strength(int n, const int* arp, const int* aci, const double* av, const int* srp,
                    const int* sci, double beta, double* sval, unsigned char* cand,
                    cudaStream_t s);
// tpos[q] = position of (j, i) in row j of the symmetric pattern S, for q = (i, j)
int launch_transpose_pos(int n, const int* srp, const int* sci, int* tpos, cudaStream_t s);
// SplitMix64 visit keys hkey[i] = splitmix64(i ^ seed)
int launch_visit_keys(int n, unsigned long long seed, unsigned long long* hkey, cudaStream_t s);
// one round of the parallel pairwise matching; commit[i] = j+2 (pair), 1 (single), 0 (wait)
int launch_match_round(int n, const int* srp, const int* sci, const int* tpos,
                       const double* sval, const unsigned char* cand,
                       const unsigned long long* hkey, const unsigned char* state, int* commit,
                       cudaStream_t s);
// apply the commits of a round; flags->count += undecided nodes left
int launch_match_apply(int n, const int* commit, unsigned char* state, int* partner,
                       DevFlags* flags, cudaStream_t s);
// rep[i] = 1 if i is the smallest member of its pair (or single)
int launch_match_reps(int n, const int* partner, int* rep, cudaStream_t s);
// agg[i] = id[min(i, partner[i])]
int launch_match_ids(int n, const int* partner, const int* id, int* agg, cudaStream_t s);
// Galerkin sums over sorted segments: out[k] = 0 + v[src[seg_start[k]]] + ... in order
int launch_segment_sums(int nseg, const int* seg_start, const int* src, const double* v,
                        double* out, cudaStream_t s);
// Sequential VerticesGrouping (Algorithms 4.1/4.2) by one warp on a symmetric graph
// whose labels are the priority ranks (degree desc, original index asc).  scratch: inV
// bitmap of ceil(n/32) words, n ints Wbar list, frontier bitmap words.  On return
// colour[r] in 1..g (by label), meta[0] = g, meta[1] = error flag (a bounded loop ran
// out).  tp/tl: the graph's two-hop lists (launch_twohop_*), or both nullptr.
// max_passes: passes of Algorithm 4.2 (colours) before the loop gives up (n always
// suffices: every pass colours at least one vertex).
int launch_colouring(int n, const int* srp, const int* sci, const int* tp, const int* tl,
                     unsigned* inV, int* wbar, unsigned* bitmap, size_t bitmap_words,
                     int* colour, int* meta, int max_passes, cudaStream_t s);

// ---- other setup kernels (setup_kernels.cu) ----
// errors in the BSR pattern: row pointers outside [0, nnz] or decreasing, unsorted / out
// of range columns, missing diagonal; ci is read only inside [0, nnz)
int launch_check_pattern(int nb, int nnz, const int* rp, const int* ci, int* dpos,
                         DevFlags* flags, cudaStream_t s);
int launch_check_finite_vals(size_t n, const double* v, DevFlags* flags, cudaStream_t s);
// MSP_ERR_PATTERN (index = permuted row) where a block couples two instances: row i of the
// permuted pattern is original row perm[i]; instance k owns the original rows
// [off[k], off[k+1])
int launch_check_block_diagonal(int nb, const int* rp, const int* ci, const int* perm, int B,
                                const int* off, DevFlags* flags, cudaStream_t s);
int launch_gather_values(size_t nnz, int bb, const int* src, const double* in, double* out,
                         cudaStream_t s);
int launch_extract_N(int b, size_t nnzb, const double* v, double* aN, cudaStream_t s);
// aN[p] <- D_N,i^-1 aN[p] for every off-diagonal block p of row i (stage N pre-scaling)
int launch_scale_N_rows(int b, int nb, const int* rp, const int* dpos, const double* dNinv,
                        double* aN, cudaStream_t s);
int launch_diag_pos(int n, const int* rp, const int* ci, int* dpos, cudaStream_t s);
// Jones-Plassmann priority keys of a symmetric graph (larger degree first, then the high
// word of SplitMix64(v ^ seed)); idx[v] = v for a stable key-value sort
int launch_jp_keys(int n, const int* srp, unsigned long long seed, unsigned long long* key,
                   int* idx, cudaStream_t s);
// one round: every uncoloured vertex whose higher-priority (smaller rank) neighbours are
// all coloured takes the smallest colour none of them has; counters[0] += vertices
// coloured, counters[1] = max(counters[1], colour)
int launch_jp_round(int n, const int* srp, const int* sci, const int* rank, int* colour,
                    int* counters, cudaStream_t s);
// two-hop lists of a graph (srp/sci): cnt[v] = sum over the neighbours k of v of deg(k),
// *total = their sum; then tl[tp[v] ...] = the neighbours' rows concatenated in row order
int launch_twohop_count(int n, const int* srp, const int* sci, int* cnt, unsigned long long* total,
                        cudaStream_t s);
int launch_twohop_fill(int n, const int* srp, const int* sci, const int* tp, int* tl,
                       cudaStream_t s);
// ELL copy (K slots per row, slot k of row i at i*K + k) of the off-diagonal entries of a
// CSR level matrix; meta[i] = count | (entries left of the diagonal) << 16, or -1 for rows
// longer than K (their slots hold (i, 0)); diag[i] = a_ii
int launch_build_ell(int n, int K, const int* rp, const int* ci, const double* v, const int* dpos,
                     int* ell_ci, double* ell_v, int* meta, double* diag, cudaStream_t s);
int launch_rdiag(int n, const int* dpos, const double* v, double* rdiag, DevFlags* flags,
                 cudaStream_t s);
// BILU(0) factorisation of the rows [r0, r1) of one colour (rows of earlier colours done)
int launch_bilu_factor(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                       double* lu, double* uinv, DevFlags* flags, cudaStream_t s);
// dense copy of a CSR matrix (n x n row-major)
int launch_csr_to_dense(int n, const int* rp, const int* ci, const double* v, double* A,
                        cudaStream_t s);
// blocked in-place Gauss-Jordan inversion of a dense n x n matrix: step k on the columns
// [j0, j1) of its panel (pivot search and row swap always over the whole matrix)
int launch_gj_pivot(int n, int k, int j0, int j1, double* A, double* col, int* piv,
                    DevFlags* flags, cudaStream_t s);
int launch_gj_update(int n, int k, int j0, int w, double* A, const double* col, cudaStream_t s);
// the steps of the panel [k0, k0 + nb) (nb <= 32) applied to every other column; T = the
// rows k0..k0+nb-1 of A (n values each) before this call
int launch_gj_panel_apply(int n, int k0, int nb, double* A, const double* T, cudaStream_t s);
int launch_gj_unscramble(int n, const int* colperm, const double* A, double* out,
                         cudaStream_t s);
int launch_cast_vals(size_t n, const double* in, float* out, cudaStream_t s);
int launch_iota(int n, int* out, cudaStream_t s);
int launch_fill_int(size_t n, int value, int* out, cudaStream_t s);
int launch_scatter_inverse(int n, const int* perm, int* iperm, cudaStream_t s);

// ---- CUB-based primitives (setup_sort.cu) ----
struct SortScratch;  // reusable temporary storage
SortScratch* sort_scratch_create();
void sort_scratch_destroy(SortScratch*);
// sort 64-bit keys ascending (stable), optional int32 payload; results in place
int sort_pairs_u64(SortScratch*, size_t n, unsigned long long* keys, int* vals, int end_bit,
                   cudaStream_t s);
int exclusive_scan_int(SortScratch*, size_t n, const int* in, int* out, cudaStream_t s);

// Symmetrised off-diagonal adjacency of a CSR/BSR pattern (Eq. adjacency-matrix).
// Allocates srp (n+1) and sci (nnz); returns nnz in *snnz.
int build_adjacency(SortScratch*, int n, const int* rp, const int* ci, int nnz,
                    DevBuf<int>& srp, DevBuf<int>& sci, int* snnz, cudaStream_t s);

}  // namespace msp

namespace msp {
// more CUB-based helpers (setup_sort.cu)
int unique_sorted_keys(SortScratch*, size_t m, unsigned long long* keys, size_t* m_out,
                       DevBuf<unsigned long long>& out, cudaStream_t s);
int rowptr_from_sorted_keys(size_t m, int n, const unsigned long long* keys, int* row_ptr,
                            cudaStream_t s);
int low32_of_keys(size_t m, const unsigned long long* keys, int* out, cudaStream_t s);
}  // namespace msp
