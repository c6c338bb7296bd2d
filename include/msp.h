/*
 * msp.h - C ABI of the GB300 (sm_103a) multi-stage preconditioned FGMRES solver.
 *
 * Operation (Zhao, Zhang, Feng, Shu, "An Improved Multi-Stage Preconditioner on GPUs
 * for Compositional Reservoir Simulation", 2022):
 *   solve A x = b for a fully implicit compositional Jacobian in block-sparse (BSR) form
 *   (Eq. Jacobian-system, Section 2.2.4) with right-preconditioned flexible GMRES(m)
 *   (Section 5: m = 30, MaxIt 1000) and the multi-stage preconditioner B of Eq. MSP,
 *   applied by Algorithm 3.1:
 *     stage N: block Gauss-Seidel on the concentration sub-system (Pi_N^T A Pi_N);
 *     stage P: quasi-IMPES decoupled restriction to pressure, UA-AMG V-cycle with
 *              pairwise aggregation, multi-colour Gauss-Seidel smoothing (PGS-MC,
 *              Algorithm 4.3, colouring by Algorithms 4.1/4.2 on the adjacency matrix
 *              of Eq. adjacency-matrix) and a dense direct coarsest solve;
 *     stage R: block ILU(0) of the whole system in colour order;
 *   with the adaptive SETUP of Section 3.2 (ASMSP): a later solve regenerates B only if
 *   the previous solve took more than mu iterations.
 *
 * Conventions (all functions):
 *   - BSR: row_ptr int32[nb+1], col_idx int32[nnzb] (ascending within a row, diagonal
 *     block present), values float64[nnzb*b*b], each block row-major (row = equation,
 *     column = unknown); unknown 0 of every block is pressure, 1..b-1 the
 *     concentrations (Eq. Jacobian-system-reservoir).  Wells are ordinary block rows.
 *   - Pointers named d_* are DEVICE pointers, h_* HOST pointers.  The library copies
 *     what it needs; the caller keeps ownership of every buffer it passes and may
 *     free it once the call returns (device work is ordered on `stream`).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device work of a
 *     call is enqueued on it; calls that return sizes or the solve info synchronise it.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Return value: MSP_OK (0), MSP_NOT_CONVERGED (1, x still valid) or a negative
 *     MSP_ERR_* code; msp_status_string() describes it.  No C++ exception crosses
 *     the ABI.  After an MSP_ERR_CUDA the handle should be freed.
 */
#ifndef MSP_GB300_H
#define MSP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSP_OK 0
#define MSP_NOT_CONVERGED 1
#define MSP_ERR_ARG (-1)
#define MSP_ERR_PATTERN (-2)
#define MSP_ERR_SINGULAR_BLOCK (-3)
#define MSP_ERR_NONFINITE (-4)
#define MSP_ERR_BREAKDOWN (-5)
#define MSP_ERR_NOMEM (-6)
#define MSP_ERR_TIMEOUT (-7)
#define MSP_ERR_CUDA (-8)

/* Preconditioner selection (msp_config.precond).  MSP_PREC_MSP is Algorithm 3.1; the
 * single-stage choices exist for testing the stages in isolation. */
#define MSP_PREC_MSP 0
#define MSP_PREC_NONE 1
#define MSP_PREC_R_ONLY 2
#define MSP_PREC_P_ONLY 3
#define MSP_PREC_N_ONLY 4

/* Arithmetic of the preconditioner (msp_config.precision).  FGMRES, its residuals,
 * orthogonalisation and Hessenberg least squares, and the coarsest dense solve are
 * always FP64. */
#define MSP_PRECISION_FP64 0
#define MSP_PRECISION_FP32 1 /* stage N/P/R values and arithmetic in FP32 */

/* Smoother of the AMG levels (msp_config.smoother); Section 5.1.1 compares the three. */
#define MSP_SMOOTHER_PGS_MC 0 /* multi-colour Gauss-Seidel, Algorithm 4.3 (the paper's) */
#define MSP_SMOOTHER_PJAC 1   /* PJAC-NO: Jacobi, all rows from the values at the start */
#define MSP_SMOOTHER_PGS_NO 2 /* PGS-NO: chunks of 16 consecutive rows swept at once, each
                               * Gauss-Seidel in order (the other chunks at their values
                               * from the start of the sweep); coarse levels uncoloured */

/* Colouring of every graph the preconditioner colours (msp_config.colouring). */
#define MSP_COLOURING_ALG41 0 /* VerticesGrouping, Algorithms 4.1/4.2 (the paper's) */
#define MSP_COLOURING_JP 1    /* greedy first-fit in Jones-Plassmann priority order (larger
                               * degree first, then the high word of SplitMix64(v ^
                               * 0x4A6F6E6573504C), then index), computed in parallel rounds;
                               * not from the paper: a faster SETUP with different colours */

typedef struct msp_handle_s* msp_handle;

typedef struct {
  int mu;          /* adaptive-setup threshold mu >= 0 (Section 3.2); 0 = plain MSP */
  int restart;     /* m of FGMRES(m), 1..64 (Section 5: 30) */
  int max_it;      /* MaxIt (Section 5: 1000) */
  int coarse_max;  /* coarsest AMG level size (Section 5: 10000) */
  int npass;       /* pairwise matching passes per AMG level (2: aggregates <= 4) */
  int pre_sweeps;  /* PGS-MC sweeps before the coarse correction (forward colours) */
  int post_sweeps; /* PGS-MC sweeps after it (backward colours) */
  int bgs_sweeps;  /* block GS sweeps of stage N, each forward in level-0 colour order,
                   * the first from zero (6; the paper fixes no count) */
  int decoupling;  /* 1 = quasi-IMPES weights omega_i = D_i^-T e_0, 0 = none */
  int bilu_order;  /* must be 0: ILU(0) in level-0 colour order */
  int precond;     /* MSP_PREC_* */
  int max_levels;  /* AMG level cap */
  double beta;     /* strong-coupling threshold of the pairwise matching (0.25) */
  unsigned long long agg_seed; /* seed of the matching visit order */
  int coarse_hard_max;         /* refuse a coarsest level larger than this */
  int precision;               /* MSP_PRECISION_* */
  int colouring;               /* MSP_COLOURING_* */
  int smoother;                /* MSP_SMOOTHER_* */
  int loop_limit; /* 0 (default): every bounded SETUP loop runs to the bound its sizes
                   * give (a colouring needs at most n passes of Algorithm 4.2, the
                   * Jones-Plassmann colouring and the pairwise matching at most n
                   * rounds).  > 0: caps each of those loops at this many passes or
                   * rounds; a loop still unfinished then returns MSP_ERR_TIMEOUT.
                   * For tests of the MSP_ERR_TIMEOUT path. */
  int autotune;   /* 1: at SETUP, time the lanes per row of the AMG levels' ELL colour
                   * sweeps and restrictions (2, 4 or 8) on the level's own data and keep
                   * the fastest; the choice is kept per (level, slots per row) for the
                   * handle's life, so later SETUPs round the same way.  0 (default): the
                   * fixed choice (one lane per 4 slots).  Changes the rounding of the
                   * sweeps' row sums, not the operator. */
} msp_config;

typedef struct {
  int status;           /* return code of the solve */
  int iterations;       /* preconditioned Arnoldi steps over all restarts (It) */
  int setup_performed;  /* 1 if this solve used a freshly generated B */
  int setup_calls;      /* SETUP calls since msp_setup (Section 3.2's SetupCalls) */
  int levels;           /* AMG levels */
  int colours_l0;       /* colours g of the level-0 (block) graph */
  double rel_residual;      /* true ||b - A x||_2 / ||b||_2 at exit */
  double rel_residual_est;  /* Arnoldi estimate at exit */
  double t_setup_ms;        /* host wall time of SETUP inside this call */
  double t_solve_ms;        /* host wall time of the Krylov solve */
} msp_solve_info;

/* Fill *cfg with the defaults above (Section 5 parameters, mu = 20).  Never fails
 * unless cfg is NULL (MSP_ERR_ARG). */
int msp_config_default(msp_config* cfg);

/* Build a solver for the BSR matrix (device arrays, see Conventions) and run SETUP:
 * adjacency matrix (Eq. adjacency-matrix), VerticesGrouping (Algorithms 4.1/4.2) and
 * the colour permutation (Algorithm 4.3 step 3) of the block graph, then the value
 * setup (decoupling, AMG hierarchy, stage-N blocks, BILU(0)).  nb >= 1, 1 <= b <= 8,
 * nnzb = row_ptr[nb].  Errors: MSP_ERR_ARG (sizes/config), MSP_ERR_PATTERN (row
 * pointers outside [0, nnzb] or decreasing, unsorted or out-of-range columns, missing
 * diagonal; col_idx is never read outside [0, nnzb)), MSP_ERR_NONFINITE, MSP_ERR_SINGULAR_BLOCK
 * (a diagonal block, its concentration sub-block, a BILU pivot or the coarsest matrix
 * is singular), MSP_ERR_NOMEM, MSP_ERR_CUDA.  On error *out is NULL. */
int msp_setup(msp_handle* out, const msp_config* cfg, int32_t nb, int32_t b,
              const int32_t* d_row_ptr, const int32_t* d_col_idx, const double* d_values,
              int64_t nnzb, void* stream);

/* New values for the same pattern (a later Newton step, Section 3.2).  Copies
 * d_values (nnzb*b*b doubles).  Does not run SETUP: the next msp_solve decides. */
int msp_update_values(msp_handle h, const double* d_values, void* stream);

/* msp_update_values with a HOST array (pinned memory gives the fastest copy). */
int msp_update_values_host(msp_handle h, const double* h_values, void* stream);

/* Values copied ahead (pipelining the host-to-device copy of the next Newton step's matrix
 * with the current solve): msp_stage_values_host enqueues the copy of h_values (HOST,
 * nnzb*b*b doubles; pinned memory makes it asynchronous; keep it valid and unchanged until
 * the copy has run) on `stream`, typically a second stream, and returns at once;
 * msp_update_values_staged then makes its own stream wait for that copy and applies the
 * values as msp_update_values does.  One staged copy at a time: staging again waits (on
 * the copy stream) until the previous staged values have been applied.
 * msp_update_values_staged without a staged copy returns MSP_ERR_ARG. */
int msp_stage_values_host(msp_handle h, const double* h_values, void* stream);
int msp_update_values_staged(msp_handle h, void* stream);

/* Solve A x = b to ||b - A x|| / ||b|| <= rel_tol with x0 = 0.  d_b, d_x: device
 * arrays of nb*b doubles (natural order; may not alias).  Runs SETUP first when the
 * adaptive rule asks for it (previous It > mu).  info may be NULL.  Returns MSP_OK,
 * MSP_NOT_CONVERGED (MaxIt reached; x holds the last iterate), MSP_ERR_NONFINITE,
 * MSP_ERR_BREAKDOWN, or a setup error.  Synchronises the stream. */
int msp_solve(msp_handle h, const double* d_b, double* d_x, double rel_tol,
              msp_solve_info* info, void* stream);

/* msp_solve with HOST arrays: copies h_b in and h_x out inside the call. */
int msp_solve_host(msp_handle h, const double* h_b, double* h_x, double rel_tol,
                   msp_solve_info* info, void* stream);

/* Release every resource of the handle (NULL is accepted). */
int msp_free(msp_handle h);

/* ---- Batched instances -------------------------------------------------------------
 * Many independent systems with one block size solved together: the caller stacks them
 * into one block-diagonal BSR matrix (instance k owns the block rows [off[k], off[k+1]),
 * and its blocks couple only rows of that range) and sets it up with msp_setup.  The
 * colouring, the aggregation, the stage operators and the coarsest direct solve of a
 * block-diagonal matrix are block diagonal, so the one preconditioner acts on every
 * instance separately; each instance then gets its own FGMRES (inner products, Hessenberg
 * matrix, convergence, restarts), while every preconditioner application, SpMV and
 * Gram-Schmidt pass is one launch over all instances. */

/* Declare the instances: count >= 1, h_row_offsets[count+1] (host) strictly increasing
 * from 0 to nb.  Errors: MSP_ERR_ARG, MSP_ERR_PATTERN (a block couples two instances). */
int msp_set_instances(msp_handle h, int32_t count, const int32_t* h_row_offsets);

/* Solve every instance to its own ||b_k - A_k x_k|| / ||b_k|| <= rel_tol (x0 = 0): d_b,
 * d_x device arrays of nb*b doubles (natural order, may not alias); h_infos (host, may be
 * NULL) receives one msp_solve_info per instance.  The adaptive rule of Section 3.2
 * regenerates the preconditioner when the largest iteration count of the previous batch
 * exceeded mu.  Each instance's FGMRES is that of msp_solve (restart m < 72) except that
 * the second Gram-Schmidt pass is always taken.  Returns MSP_OK if every instance
 * converged, else the first error status or MSP_NOT_CONVERGED; MSP_ERR_ARG if no
 * instances were declared.  Synchronises the stream. */
int msp_solve_batch(msp_handle h, const double* d_b, double* d_x, double rel_tol,
                    msp_solve_info* h_infos, void* stream);

/* Device memory the handle holds (its buffers, as allocated by the library; the CUDA
 * graph's own memory and CUDA's per-context reserves are not included). */
int msp_device_bytes(msp_handle h, int64_t* bytes);

/* Static description of a status code. */
const char* msp_status_string(int status);

/* Text of the last CUDA error seen by the calling host thread ("" if none); valid until
 * the next call on that thread.  Diagnostics only. */
const char* msp_last_error(void);

/* ---- inspection (used by the parity tests; all are exact views of solver state) ---- */

/* w = B g: one application of the configured preconditioner (Algorithm 3.1 for
 * MSP_PREC_MSP) to g; device arrays of nb*b doubles, natural order. */
int msp_apply_precond(msp_handle h, const double* d_g, double* d_w, void* stream);

/* y = A x with the current values; device arrays of nb*b doubles, natural order. */
int msp_spmv(msp_handle h, const double* d_x, double* d_y, void* stream);

/* Number of AMG levels (level 0 = the pressure matrix of the block graph). */
int msp_num_levels(msp_handle h);

/* Size, stored nonzeros and colour count of level l (0 colours: level not coloured). */
int msp_level_info(msp_handle h, int level, int32_t* n, int32_t* nnz, int32_t* ncolours);
/* Tiles of AMG level `level`: slots per row of its ELL copy (0: swept in CSR form) and the
 * lanes per row its colour sweeps and its residual restriction use (the autotuner's
 * choice with msp_config.autotune, else the fixed default).  Any output may be NULL. */
int msp_level_tiles(msp_handle h, int level, int32_t* ell_slots, int32_t* sweep_lanes,
                    int32_t* restrict_lanes);

/* Copy level l to HOST arrays (any may be NULL): perm[n] (colour-ordered index ->
 * index before colouring: the natural block row for l = 0, the aggregate number for
 * l >= 1), cptr[ncolours+1], agg[n] (index of the next level, -1 on the coarsest),
 * row_ptr[n+1], col_idx[nnz], values[nnz] of the colour-ordered level matrix. */
int msp_level_get(msp_handle h, int level, int32_t* h_perm, int32_t* h_cptr,
                  int32_t* h_agg, int32_t* h_row_ptr, int32_t* h_col_idx, double* h_values);

/* Level-0 colour (1..g) of every block row in natural order (HOST array); returns g. */
int msp_colour0(msp_handle h, int32_t* h_colour);

/* ---- launch statistics (process-wide; instrumentation for benchmarks) ----
 * mode 0: off; 1: count every kernel launch of this library; 2: also time each launch
 * of the solve phase with CUDA events recorded on its stream and add up the
 * algorithmic bytes it moves, per call site (the preconditioner then runs launch by
 * launch instead of as its CUDA graph); 3: as 2, but the preconditioner keeps running
 * as its CUDA graph, re-captured with a pair of event-record nodes around every call
 * site inside it (site "precond_graph" times each whole replay).  Timing adds two event
 * records per timed launch; in mode 3 each replay first waits for the timings of the
 * previous one.  Switching into or out of mode 3 re-captures the graph at the next
 * preconditioner application. */
int msp_stats_enable(int mode);
/* Zero all counts and timings (call-site names are kept). */
int msp_stats_reset(void);
/* Kernel launches counted since the last reset (mode >= 1). */
long long msp_stats_launches(void);
/* Number of call sites seen so far, timed or not since the last reset (waits for
 * pending timings). */
int msp_stats_count(void);
/* Call site `index`: its name (NUL-terminated, truncated to name_len), launches, summed
 * CUDA-event milliseconds, summed algorithmic bytes and summed algorithmic floating-point
 * operations (2 per FMA; recorded only at sites whose kernels can be bound by the FP64
 * rate, 0 elsewhere).  Any output may be NULL. */
int msp_stats_get(int index, char* name, int name_len, long long* launches, double* total_ms,
                  double* bytes, double* flops);

/* Measured FMA throughput of the current device (the paper has no counterpart: the
 * benchmark states the ALU ceiling of the FP64 kernels with it).  precision =
 * MSP_PRECISION_FP64 or MSP_PRECISION_FP32; *flops_per_s receives 2 x FMAs per second
 * of a kernel of independent FMA chains (8 blocks of 256 threads per SM, 8 chains of
 * 2048 steps per thread), the best of 5 launches timed with CUDA events on `stream`.
 * Allocates a small output buffer; synchronises `stream`.  MSP_ERR_ARG for another
 * precision or a NULL output. */
int msp_fma_rate(int precision, double* flops_per_s, void* stream);


/* ---- allocation-free entry point ----
 * The paper has no counterpart: this exists for callers that cannot allocate device
 * memory, e.g. code running inside a memory pool that owns the whole GPU, code that
 * must not let cudaMalloc/cudaFree synchronise the device, or environments where the
 * CUDA allocator is replaced.  It computes what msp_setup computes for the block graph
 * (the colouring returned by msp_colour0: adjacency matrix, then VerticesGrouping,
 * Algorithms 4.1/4.2) without allocating: its scratch is one fixed device array of
 * about 5.8 MB inside the library, which every GPU that loads the library holds until
 * the process exits.
 *   n               block rows, 1 <= n <= 65536 (larger: MSP_ERR_ARG, nothing runs)
 *   d_row_ptr       int32[n+1], device; row_ptr[0] = 0, row_ptr[n] - n <= 1048576
 *   d_col_idx       int32[row_ptr[n]], device; ascending within a row, diagonal present,
 *                   off-diagonal pattern structurally symmetric, <= 1023 per row
 *                   (otherwise MSP_ERR_PATTERN / MSP_ERR_ARG)
 *   d_colour        int32[n], device, output: colour 1..g of every row
 *   h_ncolours      host, output: g
 *                   Row pointers outside [0, row_ptr[n]] or decreasing give
 *                   MSP_ERR_PATTERN; col_idx is never read outside [0, row_ptr[n]).
 * Calls no cudaMalloc, cudaFree or allocating library routine.  The first call on a
 * device looks up the device address of the scratch array (cudaGetSymbolAddress), and
 * so does the first call after the device's context changed (cudaDeviceReset), so make
 * those calls before any stream capture.  Every call reuses the same array,
 * which keeps the previous call's contents: calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the caller.
 * Synchronises `stream`.  msp_noalloc_error() describes the last rejection of this
 * thread. */
int msp_vertices_grouping_noalloc(int32_t n, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                                  int32_t* d_colour, int32_t* h_ncolours, void* stream);
const char* msp_noalloc_error(void);

/* ---- Elimination of the well unknowns (Schur complement) ----------------------------
 * For the Jacobian with implicit wells [A_RR A_RW; A_WR A_WW] (Eq. Jacobian-system,
 * Section 2.2.4), stored as one BSR matrix whose last nw block rows are the wells:
 *   A_S = A_RR - A_RW A_WW^-1 A_WR       (reduced matrix on the nr = nb - nw cell rows)
 *   g_S = g_R - A_RW A_WW^-1 g_W         (msp_wells_reduce_rhs)
 *   x_W = A_WW^-1 (g_W - A_WR x_R)       (msp_wells_recover, x_R = solution of A_S)
 * Accepted layout: a cell row couples to at most one well, and a well row to no other
 * well (A_WW block diagonal); otherwise MSP_ERR_ARG.  Row c of A_S has the columns of
 * A_RR's row c, plus, where well w perforates c, the cell columns of well row w (so the
 * cells of one well become mutually coupled).  Each block is formed as
 * t = A_cw A_ww^-1, then A_RR[c,j] - t A_wj, every b x b product summed over k in order
 * without fused multiply-add, so it is reproducible bit for bit.  The reduced system is
 * then handed to msp_setup / msp_update_values / msp_solve like any other matrix. */
typedef struct msp_wells_s* msp_wells;

/* Analyse the layout, build the pattern of A_S and compute its values, A_WW^-1 and the
 * blocks the right-hand-side and recovery steps need.  nb >= 2, 1 <= b <= 8,
 * 1 <= nw < nb, nnzb = row_ptr[nb]; the pattern as for msp_setup.  Errors: MSP_ERR_ARG
 * (sizes, or a layout not accepted above), MSP_ERR_PATTERN, MSP_ERR_NONFINITE,
 * MSP_ERR_SINGULAR_BLOCK (a well's diagonal block), MSP_ERR_NOMEM, MSP_ERR_CUDA.
 * Synchronises the stream.  On error *out is NULL. */
int msp_wells_setup(msp_wells* out, int32_t nb, int32_t b, int32_t nw,
                    const int32_t* d_row_ptr, const int32_t* d_col_idx, const double* d_values,
                    int64_t nnzb, void* stream);

/* The reduced matrix: nr block rows, *nnzb blocks; row_ptr int32[nr+1], col_idx
 * int32[nnzb], values float64[nnzb*b*b] are DEVICE arrays owned by W, valid until
 * msp_wells_free; the values change with msp_wells_update_values.  Any output pointer
 * may be NULL. */
int msp_wells_reduced(msp_wells W, int32_t* nr, int64_t* nnzb, const int32_t** d_row_ptr,
                      const int32_t** d_col_idx, const double** d_values);

/* New values of the full matrix (same pattern, nnzb*b*b doubles, device): recomputes
 * A_S, A_WW^-1 and the kept blocks.  Errors: MSP_ERR_NONFINITE, MSP_ERR_SINGULAR_BLOCK,
 * MSP_ERR_CUDA.  Synchronises the stream. */
int msp_wells_update_values(msp_wells W, const double* d_values, void* stream);

/* d_gs[nr*b] = g_R - A_RW A_WW^-1 g_W for d_g[nb*b] (device; may not alias).
 * Asynchronous on `stream`. */
int msp_wells_reduce_rhs(msp_wells W, const double* d_g, double* d_gs, void* stream);

/* d_x[nb*b] = [x_R; A_WW^-1 (g_W - A_WR x_R)] with x_R = d_xs[nr*b] (device; d_x may
 * be d_xs, which must then hold nb*b doubles; d_x may not alias d_g).  The blocks of a
 * well row are taken in column order.  Asynchronous on `stream`. */
int msp_wells_recover(msp_wells W, const double* d_g, const double* d_xs, double* d_x,
                      void* stream);

/* Release W (NULL is accepted); waits for the device to finish its work. */
int msp_wells_free(msp_wells W);

/* Wells with one unknown each, as Eq. Jacobian-system has them: the bottom-hole pressure
 * of well w and its one equation.  The cell part is an ordinary BSR matrix A_RR (nr block
 * rows, b x b blocks, pattern as for msp_setup, nnzb = row_ptr[nr]); well w perforates the
 * cells well_cells[k], k in [well_ptr[w], well_ptr[w+1]) (ascending, each cell at most
 * once over all wells), with
 *   arw[k*b + r]  = A_RW: cell equation r of that cell w.r.t. the well's pressure,
 *   awr[k*b + c]  = A_WR: the well equation w.r.t. unknown c of that cell,
 *   aww[w]        = A_WW: the well equation w.r.t. its own pressure.
 * The library pads each well to a b x b block row (identity rows and columns 1..b-1, a
 * zero right-hand side there), which decouples exactly, and eliminates it as
 * msp_wells_setup does: the reduced matrix is the Schur complement of the scalar A_WW,
 * A_S[c, c'] = A_RR[c, c'] - A_RW[c] A_WR[c'] / A_WW.  All arrays are device arrays; the
 * caller keeps them.  The other msp_wells_* calls then take vectors in the padded layout
 * of nb = nr + nw block rows (msp_wells_pack_rhs / msp_wells_unpack convert).  Errors as
 * msp_wells_setup; MSP_ERR_ARG also for well_ptr not starting at 0 or decreasing, a cell
 * out of range, repeated or not ascending within its well.  Synchronises the stream. */
int msp_wells_setup_scalar(msp_wells* out, int32_t nr, int32_t b, int32_t nw,
                           const int32_t* d_row_ptr, const int32_t* d_col_idx,
                           const double* d_values, int64_t nnzb, const int32_t* d_well_ptr,
                           const int32_t* d_well_cells, const double* d_arw,
                           const double* d_awr, const double* d_aww, void* stream);

/* New values for a handle of msp_wells_setup_scalar (same pattern and perforations). */
int msp_wells_update_values_scalar(msp_wells W, const double* d_values, const double* d_arw,
                                   const double* d_awr, const double* d_aww, void* stream);

/* d_g[(nr+nw)*b] = [g_R; g_W padded with zeros] from d_gr[nr*b] and d_gw[nw] (device). */
int msp_wells_pack_rhs(msp_wells W, const double* d_gr, const double* d_gw, double* d_g,
                       void* stream);

/* d_xr[nr*b] = x_R and d_xw[nw] = the wells' pressures from a padded d_x[(nr+nw)*b]
 * (either output may be NULL). */
int msp_wells_unpack(msp_wells W, const double* d_x, double* d_xr, double* d_xw,
                     void* stream);

/* ---- Request loop (serving) -----------------------------------------------------------
 * Solves of many systems arriving over time.  A system (key) is one matrix pattern; its
 * solver handle (matrix, AMG hierarchy, stage operators) stays resident on the device
 * between requests, so the Newton steps of a reservoir reuse SETUP through the adaptive
 * rule of Section 3.2.  A pool of `slots` worker threads, each with its own CUDA stream,
 * runs admitted requests concurrently, so the work of several systems overlaps on the
 * device; a request is admitted as soon as a slot is free, its key is not busy and its
 * system fits the device-memory budget (idle resident systems are released, least
 * recently used first, to make room).  Requests of one key run one at a time in submit
 * order; requests that wait for memory for a new system keep their order among
 * themselves, while requests of resident systems (new patterns included) may pass them.  Results do not depend on the mix: every system is
 * solved by the same deterministic kernels on its own buffers. */
typedef struct msp_server_s* msp_server;

#define MSP_REQ_NEW_PATTERN 1 /* release the key's resident system and set it up again */
#define MSP_REQ_RELEASE 2     /* release the key's system after this request */

typedef struct {
  int64_t key;              /* system id */
  int32_t nb, b;            /* block rows and block size of the system */
  int64_t nnzb;             /* blocks */
  const int32_t* h_row_ptr; /* HOST pattern, read when the system is set up: the first */
  const int32_t* h_col_idx; /*   request of a key, MSP_REQ_NEW_PATTERN, or after a release */
  const double* h_values;   /* HOST nnzb*b*b values of this request's matrix; NULL keeps the
                               key's previous values */
  const double* h_rhs;      /* HOST nb*b right-hand side */
  double* h_x;              /* HOST nb*b solution (written when the request completes) */
  double rel_tol;           /* as in msp_solve */
  int32_t flags;            /* MSP_REQ_* */
} msp_request;

typedef struct {
  int64_t ticket, key;
  int32_t status;     /* as msp_solve, or the setup / update error */
  int32_t slot;       /* worker that ran it */
  int32_t setup;      /* 1: the system was set up for this request */
  int32_t pad;
  msp_solve_info info;
  double queue_ms;    /* submit -> start */
  double run_ms;      /* start -> end (setup or value update, solve, copies) */
  double latency_ms;  /* submit -> end */
  int64_t device_bytes;  /* the system's footprint after the request */
} msp_result;

typedef struct {
  int64_t submitted, completed, queued, running, rejected, evictions;
  int64_t resident_systems, resident_bytes;
  int64_t peak_charged_bytes; /* peak of the bytes charged against the budget (resident
                                 systems, and the estimates of systems being set up) */
} msp_server_stats;

/* Optional replacement of the CUDA solver as the servers' executor (tests of the
 * scheduling on hosts without a GPU, tracing).  op MSP_EXEC_RUN: run `req` on slot `slot`
 * (set the system up if `setup` is 1, else update its values), return an msp status and
 * store the system's device bytes afterwards in *device_bytes; op MSP_EXEC_RELEASE:
 * release the system of req->key.  Called from the worker threads, without the server's
 * lock held. */
#define MSP_EXEC_RUN 0
#define MSP_EXEC_RELEASE 1
typedef int (*msp_server_exec_fn)(void* user, int32_t op, const msp_request* req, int32_t slot,
                                  int32_t setup, int64_t* device_bytes);

typedef struct {
  int32_t slots;          /* worker threads / CUDA streams, 1..64 */
  int32_t device;         /* CUDA device of the workers */
  int64_t hbm_budget;     /* device bytes the resident systems may hold together */
  msp_config cfg;         /* solver configuration of every system */
  msp_server_exec_fn exec;  /* NULL: the CUDA solver */
  void* exec_user;
} msp_server_config;

/* Estimate of a solver handle's device bytes for a system of this size, used to admit a
 * system before it is set up (afterwards its measured footprint, msp_device_bytes, is
 * charged instead). */
int64_t msp_estimate_device_bytes(int32_t nb, int32_t b, int64_t nnzb, const msp_config* cfg);

/* Start the workers.  Errors: MSP_ERR_ARG (slots outside 1..64, budget <= 0, config). */
int msp_server_create(msp_server* out, const msp_server_config* cfg);

/* Queue a request; *ticket identifies it.  The host arrays must stay valid and unchanged
 * until msp_server_wait returns the ticket's result.  A request whose estimated system
 * does not fit the whole budget is completed at once with MSP_ERR_NOMEM. */
int msp_server_submit(msp_server S, const msp_request* req, int64_t* ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a ticket; on MSP_OK *res holds its
 * result and the ticket is retired.  MSP_ERR_TIMEOUT if it has not completed yet,
 * MSP_ERR_ARG for an unknown ticket. */
int msp_server_wait(msp_server S, int64_t ticket, double timeout_s, msp_result* res);

int msp_server_get_stats(msp_server S, msp_server_stats* st);

/* Finish every queued and running request, release every system, stop the workers.
 * Results not yet waited for are discarded. */
int msp_server_free(msp_server S);

#ifdef __cplusplus
}
#endif
#endif /* MSP_GB300_H */
