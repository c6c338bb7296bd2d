// Oracle: a plain, slow, single-thread FP64 implementation of the multi-stage
// preconditioned FGMRES solve of "An Improved Multi-Stage Preconditioner on GPUs for
// Compositional Reservoir Simulation" (Zhao, Zhang, Feng, Shu, 2022).
//
// THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
// baseline of the benchmark may load it.  It shares no code with the CUDA library.
//
// Every step follows the paper in order and notation; where the paper is silent the
// reading taken is stated at the step.  Compile with
// -ffp-contract=off: setup arithmetic that feeds integer decisions (the decoupling
// weights, the pressure matrix, the Galerkin sums, the strength of connection) must be
// rounded exactly as written so the CUDA path can reproduce its integer outputs.
//
// Parity pins (tests/test_oracle_*.py): colouring validity and hand traces (Alg 4.1/4.2),
// multi-colour GS vs a library triangular solve (Alg 4.3), aggregation invariants and a
// brute-force Galerkin product, AMG contraction on Poisson, ILU(0) exactness on a chain
// and its red-black closed form, Krylov finite termination, exact-preconditioner
// one-step convergence (Section 3.2), the adaptive-setup decision trace, and the full
// solve against a dense LU solution.  Against Napov-Notay's own NPAIR the aggregation is
// "parity unpinned": the paper only cites it; the oracle's reading of it is stated at
// pairwise_matching.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <tuple>
#include <map>
#include <set>
#include <utility>
#include <vector>

namespace {

enum {
  ORC_OK = 0,
  ORC_NOT_CONVERGED = 1,
  ORC_ERR_ARG = -1,
  ORC_ERR_PATTERN = -2,
  ORC_ERR_SINGULAR = -3,
  ORC_ERR_NONFINITE = -4,
  ORC_ERR_BREAKDOWN = -5,
};

enum { PREC_MSP = 0, PREC_NONE = 1, PREC_R_ONLY = 2, PREC_P_ONLY = 3, PREC_N_ONLY = 4 };

}  // namespace

extern "C" {

typedef struct {
  int mu;            // adaptive-setup threshold (Section 3.2)
  int restart;       // m of FGMRES(m)
  int max_it;        // MaxIt
  int coarse_max;    // coarsest AMG size (Section 5: 10000)
  int npass;         // pairwise matching passes per level (2: aggregates of up to 4)
  int pre_sweeps;    // PGS-MC sweeps before coarse correction (1, forward)
  int post_sweeps;   // PGS-MC sweeps after coarse correction (1, backward)
  int bgs_sweeps;    // block GS sweeps of stage N (6, each forward, from zero)
  int decoupling;    // 1 = quasi-IMPES weights (Pi_P^T unspecified), 0 = literal Pi_P^T A Pi_P
  int bilu_order;    // 0 = level-0 colour order, 1 = natural order
  int precond;       // PREC_*; 0 = MSP (Alg 3.1)
  int max_levels;    // AMG level cap
  double beta;       // strong-coupling threshold (0.25)
  unsigned long long agg_seed;  // visit-order hash seed of the pairwise matching
  int coarse_hard_max;          // refuse a coarsest level above this size
  int colouring;                // 0 = VerticesGrouping (Alg 4.1/4.2), 1 = greedy in
                                // Jones-Plassmann priority order (not the paper's)
  int smoother;                 // AMG smoother: 0 = PGS-MC, 1 = PJAC-NO, 2 = PGS-NO
} orc_config;

typedef struct {
  int status;
  int iterations;
  int setup_performed;
  int setup_calls;
  int levels;
  int colours_l0;
  double rel_residual;      // true ||b - A x|| / ||b||
  double rel_residual_est;  // Arnoldi estimate at exit
  double t_setup_ms;
  double t_solve_ms;
} orc_info;

}  // extern "C"

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

struct Csr {
  int n = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;
  int nnz() const { return (int)ci.size(); }
};

struct Bsr {
  int nb = 0, b = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;  // nnzb * b * b, row-major blocks
};

// ---------------------------------------------------------------------------------
// Adjacency matrix S of Eq. (adjacency-matrix): S_ij = 1 iff i != j and a_ij != 0.
// The paper assumes a symmetric pattern "for simplicity" (Section 4.1); the oracle
// symmetrises (S = S u S^T) so that principle (iii) holds for nonsymmetric patterns.
// Structural nonzeros count as nonzeros.  Columns sorted ascending.
// ---------------------------------------------------------------------------------
Csr adjacency(int n, const int* rp, const int* ci) {
  std::vector<std::pair<int, int>> e;
  e.reserve((size_t)2 * rp[n]);
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      if (j == i) continue;
      e.push_back({i, j});
      e.push_back({j, i});
    }
  std::sort(e.begin(), e.end());
  e.erase(std::unique(e.begin(), e.end()), e.end());
  Csr s;
  s.n = n;
  s.rp.assign(n + 1, 0);
  s.ci.resize(e.size());
  for (size_t k = 0; k < e.size(); ++k) {
    s.rp[e[k].first + 1]++;
    s.ci[k] = e[k].second;
  }
  for (int i = 0; i < n; ++i) s.rp[i + 1] += s.rp[i];
  return s;
}

// ---------------------------------------------------------------------------------
// Algorithm 4.1 (VerticesSplitting).  Inputs: the current vertex set V (in_V flags) and
// S; outputs W (an independent set, in selection order) and Wbar.  |S_i| (Table 1) is
// the degree in the full graph S.
//   "any take" a max-|S_i| vertex -> the smallest index among the maxima.
//   Wbar gets S_i restricted to V (vertices coloured earlier are not re-added).
//   The second circle of v_i is the union over k in S_i of S_k, minus S_i u {i};
//       hat S_i keeps its vertices whose colour is undetermined, i.e. that are in V.
// hat W may hold vertices that have since left V; picking one takes the else branch of
// the algorithm (it is adjacent to W), exactly as written.
// ---------------------------------------------------------------------------------
void vertices_splitting(const Csr& S, const std::vector<int>& deg, std::vector<char>& in_V,
                        std::vector<int>& W, std::vector<int>& Wbar) {
  const int n = S.n;
  typedef std::pair<int, int> Key;  // (-|S_v|, v): begin() is the max degree, smallest index
  std::set<Key> Vq, Wh;
  std::vector<char> in_W(n, 0), in_Wh(n, 0), in_Wbar(n, 0), mark(n, 0);
  for (int v = 0; v < n; ++v)
    if (in_V[v]) Vq.insert(Key(-deg[v], v));
  while (!Vq.empty()) {
    int vi = !Wh.empty() ? Wh.begin()->second : Vq.begin()->second;
    bool connected = false;
    for (int p = S.rp[vi]; p < S.rp[vi + 1]; ++p)
      if (in_W[S.ci[p]]) {
        connected = true;
        break;
      }
    if (!connected) {
      in_W[vi] = 1;
      W.push_back(vi);
      if (in_V[vi]) {
        in_V[vi] = 0;
        Vq.erase(Key(-deg[vi], vi));
      }
      if (in_Wh[vi]) {
        in_Wh[vi] = 0;
        Wh.erase(Key(-deg[vi], vi));
      }
      // Wbar = Wbar u (S_i n V),  V = V / S_i
      for (int p = S.rp[vi]; p < S.rp[vi + 1]; ++p) {
        int j = S.ci[p];
        if (in_V[j]) {
          in_V[j] = 0;
          Vq.erase(Key(-deg[j], j));
          if (!in_Wbar[j]) {
            in_Wbar[j] = 1;
            Wbar.push_back(j);
          }
        }
      }
      // hat W = hat W u hat S_i
      mark[vi] = 1;
      for (int p = S.rp[vi]; p < S.rp[vi + 1]; ++p) mark[S.ci[p]] = 1;
      for (int p = S.rp[vi]; p < S.rp[vi + 1]; ++p) {
        int k = S.ci[p];
        for (int q = S.rp[k]; q < S.rp[k + 1]; ++q) {
          int x = S.ci[q];
          if (mark[x] || !in_V[x] || in_Wh[x]) continue;
          in_Wh[x] = 1;
          Wh.insert(Key(-deg[x], x));
        }
      }
      mark[vi] = 0;
      for (int p = S.rp[vi]; p < S.rp[vi + 1]; ++p) mark[S.ci[p]] = 0;
    } else {
      if (!in_Wbar[vi]) {
        in_Wbar[vi] = 1;
        Wbar.push_back(vi);
      }
      if (in_V[vi]) {
        in_V[vi] = 0;
        Vq.erase(Key(-deg[vi], vi));
      }
      if (in_Wh[vi]) {
        in_Wh[vi] = 0;
        Wh.erase(Key(-deg[vi], vi));
      }
    }
  }
}

// Algorithm 4.2 (VerticesGrouping): repeat Algorithm 4.1 on the leftover set.
// colour[v] in 1..g, numbered in order of creation.  Returns g.
int vertices_grouping(const Csr& S, std::vector<int>& colour) {
  const int n = S.n;
  std::vector<int> deg(n);
  for (int i = 0; i < n; ++i) deg[i] = S.rp[i + 1] - S.rp[i];
  colour.assign(n, 0);
  std::vector<char> in_V(n, 1);
  int remaining = n, g = 0;
  while (remaining > 0) {
    ++g;
    std::vector<int> W, Wbar;
    vertices_splitting(S, deg, in_V, W, Wbar);
    for (int v : W) colour[v] = g;
    std::fill(in_V.begin(), in_V.end(), 0);
    for (int v : Wbar) in_V[v] = 1;
    remaining = (int)Wbar.size();
  }
  return g;
}

// Greedy first-fit colouring in Jones-Plassmann priority order: an alternative to
// Algorithms 4.1/4.2 that a GPU computes in parallel rounds with the same result
// (a vertex's colour depends only on the colours of its higher-priority neighbours).
// Priority: larger degree first, then the smaller high word of SplitMix64(v ^ seed),
// then the smaller index.  colour[v] = the smallest c >= 1 used by no higher-priority
// neighbour.  Returns the number of colours.
constexpr uint64_t kJpSeed = 0x4A6F6E6573504CULL;
uint64_t splitmix64(uint64_t x);
int jp_greedy_colouring(const Csr& S, std::vector<int>& colour) {
  const int n = S.n;
  std::vector<std::tuple<int, uint32_t, int>> order(n);
  for (int v = 0; v < n; ++v)
    order[v] = {-(S.rp[v + 1] - S.rp[v]), (uint32_t)(splitmix64((uint64_t)v ^ kJpSeed) >> 32),
                v};
  std::sort(order.begin(), order.end());
  colour.assign(n, 0);
  int g = 0;
  std::vector<int> seen(n + 2, -1);  // seen[c] == v: colour c taken around v
  for (const auto& t : order) {
    const int v = std::get<2>(t);
    for (int q = S.rp[v]; q < S.rp[v + 1]; ++q) {
      const int c = colour[S.ci[q]];  // 0 for the neighbours not coloured yet
      if (c > 0) seen[c] = v;
    }
    int c = 1;
    while (seen[c] == v) ++c;
    colour[v] = c;
    g = std::max(g, c);
  }
  return g;
}

// Colour permutation (Algorithm 4.3, step 3: the colour classes V_1..V_g become
// contiguous): perm[new] = old, stable by (colour, index); cptr[c] = first new index.
void colour_permutation(const std::vector<int>& colour, int g, std::vector<int>& perm,
                        std::vector<int>& cptr) {
  const int n = (int)colour.size();
  cptr.assign(g + 1, 0);
  for (int v = 0; v < n; ++v) cptr[colour[v]]++;
  for (int c = 0; c < g; ++c) cptr[c + 1] += cptr[c];
  std::vector<int> next(cptr.begin(), cptr.end() - 1);
  perm.resize(n);
  for (int v = 0; v < n; ++v) perm[next[colour[v] - 1]++] = v;
}

// P A P^T for a scalar CSR matrix; columns re-sorted within each row.
Csr permute_csr(const Csr& a, const std::vector<int>& perm) {
  const int n = a.n;
  std::vector<int> iperm(n);
  for (int k = 0; k < n; ++k) iperm[perm[k]] = k;
  Csr r;
  r.n = n;
  r.rp.assign(n + 1, 0);
  r.ci.reserve(a.ci.size());
  r.v.reserve(a.v.size());
  for (int k = 0; k < n; ++k) {
    int i = perm[k];
    std::vector<std::pair<int, double>> row;
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) row.push_back({iperm[a.ci[p]], a.v[p]});
    std::sort(row.begin(), row.end(),
              [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
                return x.first < y.first;
              });
    for (auto& e : row) {
      r.ci.push_back(e.first);
      r.v.push_back(e.second);
    }
    r.rp[k + 1] = (int)r.ci.size();
  }
  return r;
}

// ---------------------------------------------------------------------------------
// Small dense block helpers (b x b, row-major).  Written out plainly so the rounding is
// the textbook one.
// ---------------------------------------------------------------------------------

// Inverse by Gauss-Jordan elimination on [D | I] with partial pivoting (first maximum
// |pivot| wins).  Row operations: pivot row divided by the pivot, then every other row
// r gets row_r - a_rc * pivot_row.  Returns false on a zero pivot.
bool gj_inverse(int b, const double* D, double* X) {
  std::vector<double> a(D, D + b * b), x(b * b, 0.0);
  for (int i = 0; i < b; ++i) x[i * b + i] = 1.0;
  for (int c = 0; c < b; ++c) {
    int p = c;
    for (int r = c + 1; r < b; ++r)
      if (std::fabs(a[r * b + c]) > std::fabs(a[p * b + c])) p = r;
    if (!(a[p * b + c] != 0.0) || !std::isfinite(a[p * b + c])) return false;
    if (p != c)
      for (int k = 0; k < b; ++k) {
        std::swap(a[p * b + k], a[c * b + k]);
        std::swap(x[p * b + k], x[c * b + k]);
      }
    double piv = a[c * b + c];
    for (int k = 0; k < b; ++k) {
      a[c * b + k] = a[c * b + k] / piv;
      x[c * b + k] = x[c * b + k] / piv;
    }
    for (int r = 0; r < b; ++r) {
      if (r == c) continue;
      double f = a[r * b + c];
      for (int k = 0; k < b; ++k) {
        a[r * b + k] = a[r * b + k] - f * a[c * b + k];
        x[r * b + k] = x[r * b + k] - f * x[c * b + k];
      }
    }
  }
  std::copy(x.begin(), x.end(), X);
  return true;
}

// C = X * Y
void blk_mul(int b, const double* X, const double* Y, double* C) {
  for (int r = 0; r < b; ++r)
    for (int c = 0; c < b; ++c) {
      double s = 0.0;
      for (int m = 0; m < b; ++m) s += X[r * b + m] * Y[m * b + c];
      C[r * b + c] = s;
    }
}

// y = y - X * v   (b x b times b-vector)
void blk_gemv_sub(int b, const double* X, const double* v, double* y) {
  for (int r = 0; r < b; ++r) {
    double s = y[r];
    for (int c = 0; c < b; ++c) s -= X[r * b + c] * v[c];
    y[r] = s;
  }
}

// y = X * v
void blk_gemv(int b, const double* X, const double* v, double* y) {
  for (int r = 0; r < b; ++r) {
    double s = 0.0;
    for (int c = 0; c < b; ++c) s += X[r * b + c] * v[c];
    y[r] = s;
  }
}

// ---------------------------------------------------------------------------------
// Unsmoothed aggregation by nonsymmetric pairwise matching (Section 5 only cites NPAIR;
// the details read here):
//   strength s_ij = -(a_ij + a_ji)/2 over the symmetrised off-diagonal pattern;
//   j is a candidate of i iff s_ij >= beta * max_k s_ik and that maximum is > 0;
//   nodes are visited by ascending (splitmix64(i ^ seed), i); an unmatched node pairs
//   with its unmatched candidate of largest s_ij (ties: smaller j), else stays single;
//   aggregates are numbered by ascending smallest member.
// ---------------------------------------------------------------------------------
uint64_t splitmix64(uint64_t x) {  // Vigna's SplitMix64 output function
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double entry(const Csr& a, int i, int j) {
  auto b = a.ci.begin() + a.rp[i], e = a.ci.begin() + a.rp[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it != e && *it == j) return a.v[it - a.ci.begin()];
  return 0.0;
}

// One matching pass; returns the number of aggregates, agg[i] in [0, nagg).
int pairwise_matching(const Csr& a, double beta, uint64_t seed, std::vector<int>& agg) {
  const int n = a.n;
  Csr S = adjacency(n, a.rp.data(), a.ci.data());
  std::vector<int> cand_rp(n + 1, 0), cand;
  std::vector<double> cand_s;
  for (int i = 0; i < n; ++i) {
    double smax = 0.0;
    bool any = false;
    std::vector<double> s(S.rp[i + 1] - S.rp[i]);
    for (int p = S.rp[i]; p < S.rp[i + 1]; ++p) {
      int j = S.ci[p];
      double t = entry(a, i, j) + entry(a, j, i);
      s[p - S.rp[i]] = -0.5 * t;
      if (!any || s[p - S.rp[i]] > smax) smax = s[p - S.rp[i]];
      any = true;
    }
    if (any && smax > 0.0) {
      double thr = beta * smax;
      for (int p = S.rp[i]; p < S.rp[i + 1]; ++p)
        if (s[p - S.rp[i]] >= thr) {
          cand.push_back(S.ci[p]);
          cand_s.push_back(s[p - S.rp[i]]);
        }
    }
    cand_rp[i + 1] = (int)cand.size();
  }
  std::vector<std::pair<uint64_t, int>> order(n);
  for (int i = 0; i < n; ++i) order[i] = {splitmix64((uint64_t)i ^ seed), i};
  std::sort(order.begin(), order.end());
  std::vector<int> partner(n, -1);
  std::vector<char> marked(n, 0);
  for (int t = 0; t < n; ++t) {
    int i = order[t].second;
    if (marked[i]) continue;
    int best = -1;
    double sbest = 0.0;
    for (int p = cand_rp[i]; p < cand_rp[i + 1]; ++p) {
      int j = cand[p];
      if (marked[j]) continue;
      if (best < 0 || cand_s[p] > sbest || (cand_s[p] == sbest && j < best)) {
        best = j;
        sbest = cand_s[p];
      }
    }
    marked[i] = 1;
    if (best >= 0) {
      marked[best] = 1;
      partner[i] = best;
      partner[best] = i;
    }
  }
  agg.assign(n, -1);
  int nagg = 0;
  for (int i = 0; i < n; ++i) {
    int rep = partner[i] >= 0 ? std::min(i, partner[i]) : i;
    if (rep == i) agg[i] = nagg++;
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0) agg[i] = agg[partner[i]];
  return nagg;
}

// Galerkin product A_c = P^T A P for the 0/1 aggregation P (P_{i,agg[i]} = 1):
// A_c[I,J] = sum of a_ij over i in I, j in J; contributions added in the order of the
// fine nonzeros (rows ascending, CSR order), structural pattern (no dropping).
Csr galerkin(const Csr& a, const std::vector<int>& agg, int nc) {
  std::vector<std::map<int, double>> rows(nc);
  for (int i = 0; i < a.n; ++i) {
    int I = agg[i];
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
      int J = agg[a.ci[p]];
      auto it = rows[I].find(J);
      if (it == rows[I].end())
        rows[I][J] = 0.0 + a.v[p];
      else
        it->second = it->second + a.v[p];
    }
  }
  Csr c;
  c.n = nc;
  c.rp.assign(nc + 1, 0);
  for (int I = 0; I < nc; ++I) {
    for (auto& e : rows[I]) {
      c.ci.push_back(e.first);
      c.v.push_back(e.second);
    }
    c.rp[I + 1] = (int)c.ci.size();
  }
  return c;
}

// ---------------------------------------------------------------------------------
// Multi-colour Gauss-Seidel, Algorithm 4.3 (PGS-MC): for l = 1..g apply the classical
// GS update to every vertex of V_l.  The matrix is in colour order (colour class l is
// the index range cptr[l-1]..cptr[l]-1).  Written as the sequential sweep in colour
// order, which is what the parallel sweep computes (the vertices of one colour are
// mutually independent).  Forward = colours 1..g; backward = g..1 (the paper gives
// neither the number nor the direction of the sweeps: one forward pre-sweep and one
// backward post-sweep are taken).
// ---------------------------------------------------------------------------------
void gs_sweep(const Csr& a, const std::vector<int>& cptr, const double* b, double* x,
              bool forward) {
  const int g = (int)cptr.size() - 1;
  for (int t = 0; t < g; ++t) {
    int c = forward ? t : g - 1 - t;
    for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
      double acc = b[i], d = 0.0;
      for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
        int j = a.ci[p];
        if (j == i)
          d = a.v[p];
        else
          acc -= a.v[p] * x[j];
      }
      x[i] = acc / d;
    }
  }
}

// The smoothers the paper compares PGS-MC with (Section 5.1.1, Table 2), in natural
// (storage) order.  PJAC-NO: every row from the values at the start of the sweep.
void jacobi_sweep(const Csr& a, const double* b, double* x) {
  const std::vector<double> x0(x, x + a.n);
  for (int i = 0; i < a.n; ++i) {
    double acc = b[i], d = 0.0;
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
      const int j = a.ci[p];
      if (j == i)
        d = a.v[p];
      else
        acc -= a.v[p] * x0[j];
    }
    x[i] = acc / d;
  }
}

// PGS-NO, read as the deterministic hybrid form of a Gauss-Seidel run in parallel in
// natural order: chunks of kPgsNoChunk consecutive rows are swept at the same time,
// each in order (forward) or reverse order (backward) with its own rows' new values and
// the other rows' values from the start of the sweep.
constexpr int kPgsNoChunk = 16;
void pgs_no_sweep(const Csr& a, const double* b, double* x, bool forward) {
  const std::vector<double> x0(x, x + a.n);
  for (int c0 = 0; c0 < a.n; c0 += kPgsNoChunk) {
    const int c1 = std::min(c0 + kPgsNoChunk, a.n);
    for (int t = 0; t < c1 - c0; ++t) {
      const int i = forward ? c0 + t : c1 - 1 - t;
      double acc = b[i], d = 0.0;
      for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
        const int j = a.ci[p];
        if (j == i)
          d = a.v[p];
        else
          acc -= a.v[p] * ((j >= c0 && j < c1) ? x[j] : x0[j]);
      }
      x[i] = acc / d;
    }
  }
}

// r = b - A x
void residual_csr(const Csr& a, const double* b, const double* x, double* r) {
  for (int i = 0; i < a.n; ++i) {
    double acc = b[i];
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) acc -= a.v[p] * x[a.ci[p]];
    r[i] = acc;
  }
}

// Dense LU with partial pivoting (first maximum wins), row-major, in place.
bool dense_lu(int n, std::vector<double>& a, std::vector<int>& piv) {
  piv.resize(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    piv[c] = p;
    if (!(a[(size_t)p * n + c] != 0.0)) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) std::swap(a[(size_t)p * n + k], a[(size_t)c * n + k]);
    double d = a[(size_t)c * n + c];
    for (int r = c + 1; r < n; ++r) {
      double* ar = &a[(size_t)r * n];
      const double* ac = &a[(size_t)c * n];
      double l = ar[c] / d;
      ar[c] = l;
      for (int k = c + 1; k < n; ++k) ar[k] = ar[k] - l * ac[k];
    }
  }
  return true;
}

void dense_lu_solve(int n, const std::vector<double>& lu, const std::vector<int>& piv,
                    const double* b, double* x) {
  std::vector<double> y(b, b + n);
  for (int c = 0; c < n; ++c) std::swap(y[c], y[piv[c]]);
  for (int r = 0; r < n; ++r) {
    double s = y[r];
    for (int k = 0; k < r; ++k) s -= lu[(size_t)r * n + k] * y[k];
    y[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = y[r];
    for (int k = r + 1; k < n; ++k) s -= lu[(size_t)r * n + k] * y[k];
    y[r] = s / lu[(size_t)r * n + r];
  }
  std::copy(y.begin(), y.end(), x);
}

struct Level {
  Csr A;                  // level matrix in this level's colour order
  std::vector<int> perm;  // new -> index before colouring (aggregate id for l >= 1)
  std::vector<int> cptr;  // colour class boundaries (empty for an uncoloured level)
  std::vector<int> agg;   // fine (this level) -> coarse (next level, coloured order)
  int nc = 0;             // size of the next level
};

struct Handle {
  orc_config cfg;
  int nb = 0, b = 0;
  Bsr A0;                        // input matrix, natural order (current values)
  std::vector<int> perm0, cptr0, iperm0;  // level-0 colouring
  std::vector<int> colour0;
  int g0 = 0;
  Bsr Ap;                        // P A P^T in level-0 colour order (current values)
  std::vector<int> ap_src;       // Ap nonzero -> A0 nonzero
  // setup products (frozen between setups: on reuse only the matrix values change)
  std::vector<double> omega;     // nb * b: first row of D_i^{-1} (quasi-IMPES weights)
  std::vector<double> dN_inv;    // nb * (b-1)^2: inverses of the N diagonal sub-blocks
  std::vector<double> aN;        // nnzb * (b-1)^2: N sub-blocks of Ap at setup
  std::vector<double> lu;        // BILU(0) factors (nnzb * b * b)
  std::vector<double> u_inv;     // nb * b * b inverses of the factored pivots
  std::vector<double> u_piv;     // nb * b * b factored pivots (for tests)
  std::vector<int> bilu_perm;    // BILU row order (identity, or natural order)
  std::vector<Level> levels;
  std::vector<double> coarse_lu;
  std::vector<int> coarse_piv;
  // adaptive setup state (Section 3.2)
  int setup_calls = 0;
  int prev_it = -1;
  bool first_solve = true;
  double t_setup_ms = 0.0;
};

// ---------------------------------------------------------------------------------
// Level-0 pattern setup: adjacency, VerticesGrouping, colour permutation.
// ---------------------------------------------------------------------------------
void pattern_setup(Handle& h) {
  const int nb = h.nb, b = h.b, bb = b * b;
  Csr S = adjacency(nb, h.A0.rp.data(), h.A0.ci.data());
  h.g0 = h.cfg.colouring == 1 ? jp_greedy_colouring(S, h.colour0)
                              : vertices_grouping(S, h.colour0);
  colour_permutation(h.colour0, h.g0, h.perm0, h.cptr0);
  h.iperm0.resize(nb);
  for (int k = 0; k < nb; ++k) h.iperm0[h.perm0[k]] = k;
  // P A P^T structure, remembering where every nonzero came from
  h.Ap.nb = nb;
  h.Ap.b = b;
  h.Ap.rp.assign(nb + 1, 0);
  h.Ap.ci.clear();
  h.ap_src.clear();
  for (int k = 0; k < nb; ++k) {
    int i = h.perm0[k];
    std::vector<std::pair<int, int>> row;
    for (int p = h.A0.rp[i]; p < h.A0.rp[i + 1]; ++p) row.push_back({h.iperm0[h.A0.ci[p]], p});
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      h.Ap.ci.push_back(e.first);
      h.ap_src.push_back(e.second);
    }
    h.Ap.rp[k + 1] = (int)h.Ap.ci.size();
  }
  h.Ap.v.resize((size_t)h.Ap.ci.size() * bb);
  (void)bb;
}

void refresh_permuted_values(Handle& h) {
  const int bb = h.b * h.b;
  for (size_t q = 0; q < h.ap_src.size(); ++q)
    std::copy(&h.A0.v[(size_t)h.ap_src[q] * bb], &h.A0.v[(size_t)h.ap_src[q] * bb] + bb,
              &h.Ap.v[q * bb]);
}

int diag_pos(const Bsr& a, int i) {
  for (int p = a.rp[i]; p < a.rp[i + 1]; ++p)
    if (a.ci[p] == i) return p;
  return -1;
}

// ---------------------------------------------------------------------------------
// Value setup (SETUP of Section 3): decoupling, AMG hierarchy, BGS, BILU(0).
// ---------------------------------------------------------------------------------
int value_setup(Handle& h) {
  auto t0 = Clock::now();
  const int nb = h.nb, b = h.b, bb = b * b, bn = b - 1;
  const Bsr& A = h.Ap;
  // diagonal block inverses and quasi-IMPES weights omega_i = D_i^{-T} e_0 (the paper does
  // not specify Pi_P^T; the volume-balance row has no spatial coupling)
  std::vector<double> dinv((size_t)nb * bb);
  h.omega.assign((size_t)nb * b, 0.0);
  for (int i = 0; i < nb; ++i) {
    int p = diag_pos(A, i);
    if (!gj_inverse(b, &A.v[(size_t)p * bb], &dinv[(size_t)i * bb])) return ORC_ERR_SINGULAR;
    for (int k = 0; k < b; ++k) h.omega[(size_t)i * b + k] = dinv[(size_t)i * bb + k];
  }
  // pressure matrix A_P = Pi_P^T A Pi_P with the decoupled restriction:
  // A_P[i,j] = omega_i^T A_ij e_0  (or A_ij[0,0] without decoupling)
  Level L0;
  L0.A.n = nb;
  L0.A.rp = A.rp;
  L0.A.ci = A.ci;
  L0.A.v.resize(A.ci.size());
  for (int i = 0; i < nb; ++i)
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const double* blk = &A.v[(size_t)p * bb];
      double s;
      if (h.cfg.decoupling) {
        s = 0.0;
        for (int k = 0; k < b; ++k) s = s + h.omega[(size_t)i * b + k] * blk[k * b + 0];
      } else {
        s = blk[0];
      }
      L0.A.v[p] = s;
    }
  L0.perm.resize(nb);
  for (int i = 0; i < nb; ++i) L0.perm[i] = i;  // already in level-0 colour order
  L0.cptr = h.cptr0;
  h.levels.clear();
  h.levels.push_back(std::move(L0));
  // AMG hierarchy (Section 5: UA-AMG, NPAIR, V-cycle, coarsest size 10000, direct solve)
  for (int l = 0;; ++l) {
    Level& F = h.levels[l];
    if (F.A.n <= h.cfg.coarse_max || l + 1 >= h.cfg.max_levels) break;
    // npass pairwise passes, composed; each pass works on the previous pass's Galerkin
    // matrix; the level matrix is then formed directly from the fine matrix.
    std::vector<int> agg(F.A.n);
    for (int i = 0; i < F.A.n; ++i) agg[i] = i;
    int nc = F.A.n;
    Csr cur = F.A;
    for (int pass = 0; pass < h.cfg.npass; ++pass) {
      std::vector<int> a1;
      uint64_t seed = h.cfg.agg_seed + (uint64_t)(2 * l + pass);
      int n1 = pairwise_matching(cur, h.cfg.beta, seed, a1);
      for (int i = 0; i < F.A.n; ++i) agg[i] = a1[agg[i]];
      nc = n1;
      if (pass + 1 < h.cfg.npass) cur = galerkin(cur, a1, n1);
    }
    if ((double)nc > 0.9 * (double)F.A.n) break;  // coarsening stalled
    Csr Ac = galerkin(F.A, agg, nc);
    Level C;
    if (nc > h.cfg.coarse_max && l + 2 < h.cfg.max_levels && h.cfg.smoother != 0) {
      // PJAC-NO / PGS-NO need no colouring: natural order, one class
      C.perm.resize(nc);
      for (int i = 0; i < nc; ++i) C.perm[i] = i;
      C.cptr = {0, nc};
      C.A = std::move(Ac);
    } else if (nc > h.cfg.coarse_max && l + 2 < h.cfg.max_levels) {
      Csr Sc = adjacency(nc, Ac.rp.data(), Ac.ci.data());
      std::vector<int> colour;
      int g = h.cfg.colouring == 1 ? jp_greedy_colouring(Sc, colour)
                                   : vertices_grouping(Sc, colour);
      colour_permutation(colour, g, C.perm, C.cptr);
      C.A = permute_csr(Ac, C.perm);
    } else {
      C.perm.resize(nc);
      for (int i = 0; i < nc; ++i) C.perm[i] = i;
      C.A = std::move(Ac);
    }
    std::vector<int> ipc(nc);
    for (int k = 0; k < nc; ++k) ipc[C.perm[k]] = k;
    F.agg.resize(F.A.n);
    for (int i = 0; i < F.A.n; ++i) F.agg[i] = ipc[agg[i]];
    F.nc = nc;
    h.levels.push_back(std::move(C));
  }
  Level& Lc = h.levels.back();
  if (Lc.A.n > h.cfg.coarse_hard_max) return ORC_ERR_ARG;
  {
    const int n = Lc.A.n;
    h.coarse_lu.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int p = Lc.A.rp[i]; p < Lc.A.rp[i + 1]; ++p)
        h.coarse_lu[(size_t)i * n + Lc.A.ci[p]] = Lc.A.v[p];
    if (!dense_lu(n, h.coarse_lu, h.coarse_piv)) return ORC_ERR_SINGULAR;
  }
  // stage N: the (b-1)x(b-1) sub-blocks of Pi_N^T A Pi_N and their diagonal inverses
  if (bn > 0) {
    const size_t nnzb = A.ci.size();
    h.aN.resize(nnzb * bn * bn);
    for (size_t p = 0; p < nnzb; ++p)
      for (int r = 0; r < bn; ++r)
        for (int c = 0; c < bn; ++c) h.aN[(p * bn + r) * bn + c] = A.v[p * bb + (r + 1) * b + c + 1];
    h.dN_inv.resize((size_t)nb * bn * bn);
    for (int i = 0; i < nb; ++i) {
      int p = diag_pos(A, i);
      if (!gj_inverse(bn, &h.aN[(size_t)p * bn * bn], &h.dN_inv[(size_t)i * bn * bn]))
        return ORC_ERR_SINGULAR;
    }
  }
  // stage R: block ILU(0) on P A P^T in the level-0 colour order (fill and order are
  // not given in the paper)
  {
    h.bilu_perm.resize(nb);
    if (h.cfg.bilu_order == 0) {
      for (int i = 0; i < nb; ++i) h.bilu_perm[i] = i;
    } else {
      for (int i = 0; i < nb; ++i) h.bilu_perm[i] = h.iperm0[i];  // natural order rows
    }
    // elimination position of every row
    std::vector<int> pos(nb);
    for (int t = 0; t < nb; ++t) pos[h.bilu_perm[t]] = t;
    h.lu = A.v;
    h.u_inv.assign((size_t)nb * bb, 0.0);
    h.u_piv.assign((size_t)nb * bb, 0.0);
    std::vector<double> L(bb), tmp(bb);
    for (int t = 0; t < nb; ++t) {
      int i = h.bilu_perm[t];
      // entries of row i ordered by elimination position of their column
      std::vector<std::pair<int, int>> row;
      for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) row.push_back({pos[A.ci[p]], p});
      std::sort(row.begin(), row.end());
      for (size_t e = 0; e < row.size(); ++e) {
        if (row[e].first >= t) break;
        int p = row[e].second, k = A.ci[p];
        blk_mul(b, &h.lu[(size_t)p * bb], &h.u_inv[(size_t)k * bb], L.data());
        std::copy(L.begin(), L.end(), &h.lu[(size_t)p * bb]);
        for (size_t f = e + 1; f < row.size(); ++f) {
          int q = row[f].second, j = A.ci[q];
          // (k, j) in the pattern?
          int r = -1;
          for (int s = A.rp[k]; s < A.rp[k + 1]; ++s)
            if (A.ci[s] == j) {
              r = s;
              break;
            }
          if (r < 0) continue;
          blk_mul(b, L.data(), &h.lu[(size_t)r * bb], tmp.data());
          for (int m = 0; m < bb; ++m) h.lu[(size_t)q * bb + m] -= tmp[m];
        }
      }
      int d = diag_pos(A, i);
      std::copy(&h.lu[(size_t)d * bb], &h.lu[(size_t)d * bb] + bb, &h.u_piv[(size_t)i * bb]);
      if (!gj_inverse(b, &h.lu[(size_t)d * bb], &h.u_inv[(size_t)i * bb])) return ORC_ERR_SINGULAR;
    }
  }
  h.setup_calls++;
  h.t_setup_ms += ms_since(t0);
  return ORC_OK;
}

// ---------------------------------------------------------------------------------
// Preconditioner application (all vectors in level-0 colour order, length nb*b)
// ---------------------------------------------------------------------------------
void bsr_residual(const Bsr& a, const double* g, const double* w, double* r) {
  const int b = a.b, bb = b * b;
  for (int i = 0; i < a.nb; ++i) {
    std::vector<double> acc(g + (size_t)i * b, g + (size_t)i * b + b);
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p)
      blk_gemv_sub(b, &a.v[(size_t)p * bb], w + (size_t)a.ci[p] * b, acc.data());
    std::copy(acc.begin(), acc.end(), r + (size_t)i * b);
  }
}

void bsr_spmv(const Bsr& a, const double* x, double* y) {
  const int b = a.b, bb = b * b;
  std::vector<double> t(b);
  for (int i = 0; i < a.nb; ++i) {
    for (int r = 0; r < b; ++r) y[(size_t)i * b + r] = 0.0;
    for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
      blk_gemv(b, &a.v[(size_t)p * bb], x + (size_t)a.ci[p] * b, t.data());
      for (int r = 0; r < b; ++r) y[(size_t)i * b + r] += t[r];
    }
  }
}

// V-cycle on level l: x = B_l b (x starts at zero), Section 5 settings; one forward pre-
// and one backward post-sweep, coarse correction added unscaled (not given in the paper).
void vcycle(const Handle& h, int l, const double* b, double* x) {
  const Level& L = h.levels[l];
  const int n = L.A.n;
  if (l + 1 == (int)h.levels.size()) {
    dense_lu_solve(n, h.coarse_lu, h.coarse_piv, b, x);
    return;
  }
  auto smooth = [&](bool forward) {
    if (h.cfg.smoother == 1)
      jacobi_sweep(L.A, b, x);
    else if (h.cfg.smoother == 2)
      pgs_no_sweep(L.A, b, x, forward);
    else
      gs_sweep(L.A, L.cptr, b, x, forward);
  };
  std::fill(x, x + n, 0.0);
  for (int s = 0; s < h.cfg.pre_sweeps; ++s) smooth(true);
  std::vector<double> r(n), bc(L.nc, 0.0), xc(L.nc);
  residual_csr(L.A, b, x, r.data());
  for (int i = 0; i < n; ++i) bc[L.agg[i]] += r[i];  // restriction P^T r
  vcycle(h, l + 1, bc.data(), xc.data());
  for (int i = 0; i < n; ++i) x[i] += xc[L.agg[i]];  // prolongation by injection
  for (int s = 0; s < h.cfg.post_sweeps; ++s) smooth(false);
}

// w += Pi_N B_N Pi_N^T r : block GS on the (b-1)x(b-1) sub-blocks, colour order, x0 = 0.
// Eq. MSP names block Gauss-Seidel for B_N without a number of sweeps; bgs_sweeps forward
// sweeps are taken (default 6: B_N is then close enough to the inverse of the
// concentration block that stage N stops limiting the convergence on elliptic-like
// concentration couplings)
void stage_N(const Handle& h, const double* r, double* w) {
  const int nb = h.nb, b = h.b, bn = b - 1;
  if (bn <= 0) return;
  const Bsr& A = h.Ap;
  std::vector<double> x((size_t)nb * bn, 0.0), acc(bn);
  for (int s = 0; s < h.cfg.bgs_sweeps; ++s)
    for (int c = 0; c < h.g0; ++c)
      for (int i = h.cptr0[c]; i < h.cptr0[c + 1]; ++i) {
        for (int k = 0; k < bn; ++k) acc[k] = r[(size_t)i * b + k + 1];
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
          int j = A.ci[p];
          if (j == i) continue;
          blk_gemv_sub(bn, &h.aN[(size_t)p * bn * bn], &x[(size_t)j * bn], acc.data());
        }
        blk_gemv(bn, &h.dN_inv[(size_t)i * bn * bn], acc.data(), &x[(size_t)i * bn]);
      }
  for (int i = 0; i < nb; ++i)
    for (int k = 0; k < bn; ++k) w[(size_t)i * b + k + 1] += x[(size_t)i * bn + k];
}

// w += Pi_P B_P Pi_P^T r
void stage_P(const Handle& h, const double* r, double* w) {
  const int nb = h.nb, b = h.b;
  std::vector<double> rp(nb), ep(nb);
  for (int i = 0; i < nb; ++i) {
    if (h.cfg.decoupling) {
      double s = 0.0;
      for (int k = 0; k < b; ++k) s = s + h.omega[(size_t)i * b + k] * r[(size_t)i * b + k];
      rp[i] = s;
    } else {
      rp[i] = r[(size_t)i * b];
    }
  }
  vcycle(h, 0, rp.data(), ep.data());
  for (int i = 0; i < nb; ++i) w[(size_t)i * b] += ep[i];
}

// w += R r : block ILU(0) forward (unit lower) and backward substitution
void stage_R(const Handle& h, const double* r, double* w) {
  const int nb = h.nb, b = h.b, bb = b * b;
  const Bsr& A = h.Ap;
  std::vector<int> pos(nb);
  for (int t = 0; t < nb; ++t) pos[h.bilu_perm[t]] = t;
  std::vector<double> y((size_t)nb * b), acc(b);
  for (int t = 0; t < nb; ++t) {
    int i = h.bilu_perm[t];
    for (int k = 0; k < b; ++k) acc[k] = r[(size_t)i * b + k];
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      int j = A.ci[p];
      if (pos[j] < t) blk_gemv_sub(b, &h.lu[(size_t)p * bb], &y[(size_t)j * b], acc.data());
    }
    std::copy(acc.begin(), acc.end(), &y[(size_t)i * b]);
  }
  std::vector<double> x((size_t)nb * b);
  for (int t = nb - 1; t >= 0; --t) {
    int i = h.bilu_perm[t];
    for (int k = 0; k < b; ++k) acc[k] = y[(size_t)i * b + k];
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      int j = A.ci[p];
      if (pos[j] > t) blk_gemv_sub(b, &h.lu[(size_t)p * bb], &x[(size_t)j * b], acc.data());
    }
    blk_gemv(b, &h.u_inv[(size_t)i * bb], acc.data(), &x[(size_t)i * b]);
  }
  for (size_t k = 0; k < (size_t)nb * b; ++k) w[k] += x[k];
}

// Algorithm 3.1 (MSP preconditioning), w = B g, w starting at zero; A is the current
// matrix, the stage operators come from the last setup (Section 3.2 reuses the
// preconditioner, not the matrix: the residual steps use the current A).
void apply_precond(const Handle& h, const double* g, double* w) {
  const size_t n = (size_t)h.nb * h.b;
  std::fill(w, w + n, 0.0);
  std::vector<double> r(n);
  switch (h.cfg.precond) {
    case PREC_NONE:
      std::copy(g, g + n, w);
      return;
    case PREC_R_ONLY:
      stage_R(h, g, w);
      return;
    case PREC_P_ONLY:
      stage_P(h, g, w);
      return;
    case PREC_N_ONLY:
      stage_N(h, g, w);
      return;
    default:
      break;
  }
  bsr_residual(h.Ap, g, w, r.data());  // r = g - A w
  stage_N(h, r.data(), w);             // w = w + Pi_N B_N Pi_N^T r
  bsr_residual(h.Ap, g, w, r.data());  // r = g - A w
  stage_P(h, r.data(), w);             // w = w + Pi_P B_P Pi_P^T r
  bsr_residual(h.Ap, g, w, r.data());  // r = g - A w
  stage_R(h, r.data(), w);             // w = w + R r
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t k = 0; k < a.size(); ++k) s += a[k] * b[k];
  return s;
}

// ---------------------------------------------------------------------------------
// Right-preconditioned flexible GMRES(m) (Section 5: m = 30, MaxIt 1000), modified
// Gram-Schmidt, Givens rotations, x0 = 0.  Converged when the Arnoldi estimate of
// ||b - A x|| / ||b|| is <= tol and the true residual confirms it at the cycle end.
// All vectors in level-0 colour order.
// ---------------------------------------------------------------------------------
int fgmres(const Handle& h, const double* bvec, double* xout, double tol, int* iters,
           double* relres, double* relres_est) {
  const size_t n = (size_t)h.nb * h.b;
  const int m = h.cfg.restart;
  std::vector<double> b(bvec, bvec + n), x(n, 0.0), r(n);
  double bnorm = std::sqrt(dot(b, b));
  *iters = 0;
  *relres = 0.0;
  *relres_est = 0.0;
  if (!std::isfinite(bnorm)) return ORC_ERR_NONFINITE;
  if (bnorm == 0.0) {
    std::fill(xout, xout + n, 0.0);
    return ORC_OK;
  }
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), s(m + 1);
  int it = 0, status = ORC_NOT_CONVERGED;
  double est = 1.0;
  while (true) {
    bsr_residual(h.Ap, b.data(), x.data(), r.data());
    double beta = std::sqrt(dot(r, r));
    if (!std::isfinite(beta)) return ORC_ERR_NONFINITE;
    if (beta / bnorm <= tol) {
      est = beta / bnorm;
      status = ORC_OK;
      break;
    }
    if (it >= h.cfg.max_it) break;
    for (size_t k = 0; k < n; ++k) V[0][k] = r[k] / beta;
    std::fill(s.begin(), s.end(), 0.0);
    s[0] = beta;
    int j_used = 0;
    bool breakdown = false;
    for (int j = 0; j < m; ++j) {
      apply_precond(h, V[j].data(), Z[j].data());
      bsr_spmv(h.Ap, Z[j].data(), V[j + 1].data());
      ++it;
      for (int i = 0; i <= j; ++i) {
        double hij = dot(V[j + 1], V[i]);
        H[(size_t)i * m + j] = hij;
        for (size_t k = 0; k < n; ++k) V[j + 1][k] -= hij * V[i][k];
      }
      double hn = std::sqrt(dot(V[j + 1], V[j + 1]));
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (size_t k = 0; k < n; ++k) V[j + 1][k] /= hn;
      // apply the previous rotations to column j, then a new one to zero H[j+1][j]
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      double rho = std::sqrt(a * a + c * c);
      if (rho == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
      } else {
        cs[j] = a / rho;
        sn[j] = c / rho;
      }
      H[(size_t)j * m + j] = rho;
      H[(size_t)(j + 1) * m + j] = 0.0;
      s[j + 1] = -sn[j] * s[j];
      s[j] = cs[j] * s[j];
      j_used = j + 1;
      est = std::fabs(s[j + 1]) / bnorm;
      if (!std::isfinite(est)) return ORC_ERR_NONFINITE;
      if (hn == 0.0) breakdown = true;
      if (est <= tol || it >= h.cfg.max_it || breakdown) break;
    }
    // y = H^{-1} s (upper triangular), x = x + Z y
    std::vector<double> y(j_used);
    for (int i = j_used - 1; i >= 0; --i) {
      double t = s[i];
      for (int k = i + 1; k < j_used; ++k) t -= H[(size_t)i * m + k] * y[k];
      y[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
    }
    for (int k = 0; k < j_used; ++k)
      for (size_t q = 0; q < n; ++q) x[q] += y[k] * Z[k][q];
    if (breakdown) {
      bsr_residual(h.Ap, b.data(), x.data(), r.data());
      double rr = std::sqrt(dot(r, r)) / bnorm;
      if (!(rr <= tol)) {
        *iters = it;
        *relres = rr;
        *relres_est = est;
        std::copy(x.begin(), x.end(), xout);
        return ORC_ERR_BREAKDOWN;
      }
    }
  }
  bsr_residual(h.Ap, b.data(), x.data(), r.data());
  *relres = std::sqrt(dot(r, r)) / bnorm;
  *relres_est = est;
  *iters = it;
  std::copy(x.begin(), x.end(), xout);
  return status;
}

bool all_finite(const double* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

int check_pattern(int nb, const int* rp, const int* ci) {
  if (rp[0] != 0) return ORC_ERR_PATTERN;
  for (int i = 0; i < nb; ++i) {
    if (rp[i + 1] < rp[i]) return ORC_ERR_PATTERN;
    bool diag = false;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= nb) return ORC_ERR_PATTERN;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return ORC_ERR_PATTERN;
      if (ci[p] == i) diag = true;
    }
    if (!diag) return ORC_ERR_PATTERN;
  }
  return ORC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Eliminating the well unknowns (Eq. Jacobian-system: reservoir rows R first, well rows
// W last): the Schur complement A_S = A_RR - A_RW A_WW^{-1} A_WR on the reservoir rows,
// the right-hand side g_R - A_RW A_WW^{-1} g_W, and afterwards
// x_W = A_WW^{-1} (g_W - A_WR x_R).  A_WW must be block diagonal (wells not coupled to
// each other) and every reservoir row may couple to one well at most.
// ---------------------------------------------------------------------------------
struct Wells {
  int nb = 0, b = 0, nw = 0, nr = 0;  // block rows: all, wells (the last nw), reservoir
  Bsr A;                              // the full matrix (current values)
  Bsr S;                              // the reduced matrix on the reservoir rows
  std::vector<double> winv;           // nw b x b: A_WW^{-1}
  std::vector<int> well_of, cw_pos;   // reservoir row -> its well and the A_RW block, or -1
  // per reduced nonzero: the A_RR block (or -1), the well (or -1), the A_RW and A_WR blocks
  std::vector<int> s_orig, s_well, s_cw, s_wc;
};

int find_block(const Bsr& A, int i, int j) {
  const auto b0 = A.ci.begin() + A.rp[i], b1 = A.ci.begin() + A.rp[i + 1];
  const auto it = std::lower_bound(b0, b1, j);
  return (it != b1 && *it == j) ? (int)(it - A.ci.begin()) : -1;
}

int wells_values(Wells& W) {
  const int b = W.b, bb = b * b;
  for (int w = 0; w < W.nw; ++w) {
    const int r = W.nr + w, pd = find_block(W.A, r, r);
    if (pd < 0 || !gj_inverse(b, &W.A.v[(size_t)pd * bb], &W.winv[(size_t)w * bb]))
      return ORC_ERR_SINGULAR;
  }
  std::vector<double> t(bb);
  for (size_t p = 0; p < W.s_orig.size(); ++p) {
    double* out = &W.S.v[p * bb];
    for (int k = 0; k < bb; ++k) out[k] = W.s_orig[p] >= 0 ? W.A.v[(size_t)W.s_orig[p] * bb + k] : 0.0;
    if (W.s_well[p] < 0) continue;
    const double* acw = &W.A.v[(size_t)W.s_cw[p] * bb];
    const double* wi = &W.winv[(size_t)W.s_well[p] * bb];
    const double* awc = &W.A.v[(size_t)W.s_wc[p] * bb];
    for (int r = 0; r < b; ++r)  // t = A_RW A_WW^{-1}
      for (int c = 0; c < b; ++c) {
        double acc = 0.0;
        for (int k = 0; k < b; ++k) acc += acw[r * b + k] * wi[k * b + c];
        t[r * b + c] = acc;
      }
    for (int r = 0; r < b; ++r)  // out -= t A_WR
      for (int c = 0; c < b; ++c) {
        double acc = 0.0;
        for (int k = 0; k < b; ++k) acc += t[r * b + k] * awc[k * b + c];
        out[r * b + c] -= acc;
      }
  }
  return ORC_OK;
}

int wells_build(Wells& W) {
  const int nr = W.nr;
  const Bsr& A = W.A;
  W.well_of.assign(nr, -1);
  W.cw_pos.assign(nr, -1);
  for (int i = 0; i < W.nb; ++i)
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int j = A.ci[p];
      if (i >= nr && j >= nr && j != i) return ORC_ERR_ARG;  // wells coupled to each other
      if (i < nr && j >= nr) {
        if (W.well_of[i] >= 0) return ORC_ERR_ARG;  // a second well on one cell
        W.well_of[i] = j - nr;
        W.cw_pos[i] = p;
      }
    }
  W.S.nb = nr;
  W.S.b = W.b;
  W.S.rp.assign(nr + 1, 0);
  W.S.ci.clear();
  W.s_orig.clear();
  W.s_well.clear();
  W.s_cw.clear();
  W.s_wc.clear();
  for (int c = 0; c < nr; ++c) {
    std::vector<int> cols;
    for (int p = A.rp[c]; p < A.rp[c + 1]; ++p)
      if (A.ci[p] < nr) cols.push_back(A.ci[p]);
    const int w = W.well_of[c];
    if (w >= 0)
      for (int p = A.rp[nr + w]; p < A.rp[nr + w + 1]; ++p)
        if (A.ci[p] < nr) cols.push_back(A.ci[p]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (int j : cols) {
      W.S.ci.push_back(j);
      W.s_orig.push_back(find_block(A, c, j));
      const int wc = w >= 0 ? find_block(A, nr + w, j) : -1;
      W.s_well.push_back(wc >= 0 ? w : -1);
      W.s_cw.push_back(wc >= 0 ? W.cw_pos[c] : -1);
      W.s_wc.push_back(wc);
    }
    W.S.rp[c + 1] = (int)W.S.ci.size();
  }
  W.S.v.assign(W.S.ci.size() * (size_t)W.b * W.b, 0.0);
  W.winv.assign((size_t)W.nw * W.b * W.b, 0.0);
  return wells_values(W);
}


// =================================================================================
// C interface (ctypes)
// =================================================================================
extern "C" {

void orc_config_default(orc_config* c) {
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
  c->precond = PREC_MSP;
  c->max_levels = 20;
  c->beta = 0.25;
  c->agg_seed = 0x2208085940ULL;
  c->coarse_hard_max = 20000;
  c->colouring = 0;
  c->smoother = 0;
}

void* orc_create(const orc_config* cfg, int nb, int b, const int* rp, const int* ci,
                 const double* v, int* status) {
  *status = ORC_OK;
  if (nb <= 0 || b <= 0 || b > 16 || !cfg) {
    *status = ORC_ERR_ARG;
    return nullptr;
  }
  int st = check_pattern(nb, rp, ci);
  if (st != ORC_OK) {
    *status = st;
    return nullptr;
  }
  const size_t nnzb = (size_t)rp[nb];
  if (!all_finite(v, nnzb * b * b)) {
    *status = ORC_ERR_NONFINITE;
    return nullptr;
  }
  Handle* h = new Handle();
  h->cfg = *cfg;
  h->nb = nb;
  h->b = b;
  h->A0.nb = nb;
  h->A0.b = b;
  h->A0.rp.assign(rp, rp + nb + 1);
  h->A0.ci.assign(ci, ci + nnzb);
  h->A0.v.assign(v, v + nnzb * b * b);
  auto t0 = Clock::now();
  pattern_setup(*h);
  h->t_setup_ms += ms_since(t0);
  refresh_permuted_values(*h);
  st = value_setup(*h);  // iota = 1: the preconditioner is generated
  if (st != ORC_OK) {
    *status = st;
    delete h;
    return nullptr;
  }
  return h;
}

void orc_free(void* p) { delete static_cast<Handle*>(p); }

// New values for the same pattern (a later Newton step).  Does not run SETUP: the
// adaptive rule decides at the next solve (Section 3.2).
int orc_update_values(void* p, const double* v) {
  Handle* h = static_cast<Handle*>(p);
  const size_t cnt = h->A0.v.size();
  if (!all_finite(v, cnt)) return ORC_ERR_NONFINITE;
  std::copy(v, v + cnt, h->A0.v.begin());
  refresh_permuted_values(*h);
  return ORC_OK;
}

// Solve A x = b (natural ordering in and out) with the adaptive setup of Section 3.2:
// at a later solve iota the preconditioner is regenerated iff It^(iota-1) > mu.
int orc_solve(void* p, const double* rhs, double* x, double tol, orc_info* info) {
  Handle* h = static_cast<Handle*>(p);
  const int nb = h->nb, b = h->b;
  std::memset(info, 0, sizeof(orc_info));
  if (!all_finite(rhs, (size_t)nb * b)) {
    info->status = ORC_ERR_NONFINITE;
    return ORC_ERR_NONFINITE;
  }
  double tsetup0 = h->t_setup_ms;
  if (!h->first_solve && h->prev_it > h->cfg.mu) {
    int st = value_setup(*h);
    if (st != ORC_OK) {
      info->status = st;
      return st;
    }
    info->setup_performed = 1;
  } else if (h->first_solve) {
    info->setup_performed = 1;  // generated at creation (iota = 1)
  }
  h->first_solve = false;
  auto t0 = Clock::now();
  std::vector<double> bp((size_t)nb * b), xp((size_t)nb * b);
  for (int k = 0; k < nb; ++k)
    for (int r = 0; r < b; ++r) bp[(size_t)k * b + r] = rhs[(size_t)h->perm0[k] * b + r];
  int it = 0;
  double rr = 0.0, est = 0.0;
  int st = fgmres(*h, bp.data(), xp.data(), tol, &it, &rr, &est);
  for (int k = 0; k < nb; ++k)
    for (int r = 0; r < b; ++r) x[(size_t)h->perm0[k] * b + r] = xp[(size_t)k * b + r];
  h->prev_it = it;
  info->status = st;
  info->iterations = it;
  info->setup_calls = h->setup_calls;
  info->levels = (int)h->levels.size();
  info->colours_l0 = h->g0;
  info->rel_residual = rr;
  info->rel_residual_est = est;
  info->t_setup_ms = h->t_setup_ms - tsetup0;
  info->t_solve_ms = ms_since(t0);
  return st;
}

// w = B g for the configured preconditioner (natural ordering in and out).
int orc_apply_precond(void* p, const double* g, double* w) {
  Handle* h = static_cast<Handle*>(p);
  const int nb = h->nb, b = h->b;
  std::vector<double> gp((size_t)nb * b), wp((size_t)nb * b);
  for (int k = 0; k < nb; ++k)
    for (int r = 0; r < b; ++r) gp[(size_t)k * b + r] = g[(size_t)h->perm0[k] * b + r];
  apply_precond(*h, gp.data(), wp.data());
  for (int k = 0; k < nb; ++k)
    for (int r = 0; r < b; ++r) w[(size_t)h->perm0[k] * b + r] = wp[(size_t)k * b + r];
  return ORC_OK;
}

// y = A x with the current values (natural ordering).
int orc_spmv(void* p, const double* x, double* y) {
  Handle* h = static_cast<Handle*>(p);
  bsr_spmv(h->A0, x, y);
  return ORC_OK;
}

// Change MaxIt of later solves (the CPU baseline times single Arnoldi steps).
int orc_set_max_it(void* p, int max_it) {
  if (max_it < 0) return ORC_ERR_ARG;
  static_cast<Handle*>(p)->cfg.max_it = max_it;
  return ORC_OK;
}

int orc_num_levels(void* p) { return (int)static_cast<Handle*>(p)->levels.size(); }
int orc_colours_l0(void* p) { return static_cast<Handle*>(p)->g0; }
int orc_setup_calls(void* p) { return static_cast<Handle*>(p)->setup_calls; }

// size, nonzeros and colour count of level l (colour count 0: level not coloured)
int orc_level_info(void* p, int l, int* n, int* nnz, int* ncolours) {
  Handle* h = static_cast<Handle*>(p);
  if (l < 0 || l >= (int)h->levels.size()) return ORC_ERR_ARG;
  const Level& L = h->levels[l];
  *n = L.A.n;
  *nnz = L.A.nnz();
  *ncolours = L.cptr.empty() ? 0 : (int)L.cptr.size() - 1;
  return ORC_OK;
}

// perm (new -> old), colour class pointers, aggregation map (to the next level's
// colour-ordered index, -1 entries on the coarsest level) and the level matrix.
int orc_level_get(void* p, int l, int* perm, int* cptr, int* agg, int* rp, int* ci,
                  double* v) {
  Handle* h = static_cast<Handle*>(p);
  if (l < 0 || l >= (int)h->levels.size()) return ORC_ERR_ARG;
  const Level& L = h->levels[l];
  if (l == 0) {
    if (perm) std::copy(h->perm0.begin(), h->perm0.end(), perm);
  } else if (perm) {
    std::copy(L.perm.begin(), L.perm.end(), perm);
  }
  if (cptr) std::copy(L.cptr.begin(), L.cptr.end(), cptr);
  if (agg) {
    if (L.agg.empty())
      std::fill(agg, agg + L.A.n, -1);
    else
      std::copy(L.agg.begin(), L.agg.end(), agg);
  }
  if (rp) std::copy(L.A.rp.begin(), L.A.rp.end(), rp);
  if (ci) std::copy(L.A.ci.begin(), L.A.ci.end(), ci);
  if (v) std::copy(L.A.v.begin(), L.A.v.end(), v);
  return ORC_OK;
}

// level-0 colour of every block row (natural index), 1..g
int orc_colour0(void* p, int* colour) {
  Handle* h = static_cast<Handle*>(p);
  std::copy(h->colour0.begin(), h->colour0.end(), colour);
  return h->g0;
}

// factored BILU pivot blocks (before inversion), colour order
int orc_bilu_pivots(void* p, double* out) {
  Handle* h = static_cast<Handle*>(p);
  std::copy(h->u_piv.begin(), h->u_piv.end(), out);
  return ORC_OK;
}

// Standalone Algorithm 4.2 on a pattern: colour[v] in 1..g; returns g.
// Standalone PJAC-NO / PGS-NO sweeps on a CSR matrix (x updated in place).
void orc_jacobi_sweep(int n, const int* rp, const int* ci, const double* v, const double* b,
                      double* x) {
  Csr a;
  a.n = n;
  a.rp.assign(rp, rp + n + 1);
  a.ci.assign(ci, ci + rp[n]);
  a.v.assign(v, v + rp[n]);
  jacobi_sweep(a, b, x);
}

void orc_pgs_no_sweep(int n, const int* rp, const int* ci, const double* v, const double* b,
                      double* x, int forward) {
  Csr a;
  a.n = n;
  a.rp.assign(rp, rp + n + 1);
  a.ci.assign(ci, ci + rp[n]);
  a.v.assign(v, v + rp[n]);
  pgs_no_sweep(a, b, x, forward != 0);
}

void* orc_wells_create(int nb, int b, int nw, const int* rp, const int* ci, const double* v,
                       int* status) {
  *status = ORC_OK;
  if (nb <= 0 || b <= 0 || nw < 1 || nw >= nb) {
    *status = ORC_ERR_ARG;
    return nullptr;
  }
  if ((*status = check_pattern(nb, rp, ci)) != ORC_OK) return nullptr;
  auto* W = new Wells();
  W->nb = nb;
  W->b = b;
  W->nw = nw;
  W->nr = nb - nw;
  W->A.nb = nb;
  W->A.b = b;
  W->A.rp.assign(rp, rp + nb + 1);
  W->A.ci.assign(ci, ci + rp[nb]);
  W->A.v.assign(v, v + (size_t)rp[nb] * b * b);
  *status = wells_build(*W);
  if (*status != ORC_OK) {
    delete W;
    return nullptr;
  }
  return W;
}

void orc_wells_free(void* h) { delete static_cast<Wells*>(h); }

int orc_wells_nnzb(void* h) { return (int)static_cast<Wells*>(h)->S.ci.size(); }

void orc_wells_get(void* h, int* rp, int* ci, double* v) {
  const Wells& W = *static_cast<Wells*>(h);
  std::copy(W.S.rp.begin(), W.S.rp.end(), rp);
  std::copy(W.S.ci.begin(), W.S.ci.end(), ci);
  std::copy(W.S.v.begin(), W.S.v.end(), v);
}

int orc_wells_update_values(void* h, const double* v) {
  Wells& W = *static_cast<Wells*>(h);
  std::copy(v, v + W.A.v.size(), W.A.v.begin());
  return wells_values(W);
}

// gs = g_R - A_RW A_WW^{-1} g_W
void orc_wells_reduce_rhs(void* h, const double* g, double* gs) {
  const Wells& W = *static_cast<Wells*>(h);
  const int b = W.b, bb = b * b;
  std::vector<double> y(b);
  for (int c = 0; c < W.nr; ++c) {
    for (int k = 0; k < b; ++k) gs[(size_t)c * b + k] = g[(size_t)c * b + k];
    const int w = W.well_of[c];
    if (w < 0) continue;
    const double* wi = &W.winv[(size_t)w * bb];
    const double* gw = &g[(size_t)(W.nr + w) * b];
    for (int r = 0; r < b; ++r) {
      double acc = 0.0;
      for (int k = 0; k < b; ++k) acc += wi[r * b + k] * gw[k];
      y[r] = acc;
    }
    const double* acw = &W.A.v[(size_t)W.cw_pos[c] * bb];
    for (int r = 0; r < b; ++r) {
      double acc = 0.0;
      for (int k = 0; k < b; ++k) acc += acw[r * b + k] * y[k];
      gs[(size_t)c * b + r] -= acc;
    }
  }
}

// x_R = xs; x_W = A_WW^{-1} (g_W - A_WR x_R)
void orc_wells_recover(void* h, const double* g, const double* xs, double* x) {
  const Wells& W = *static_cast<Wells*>(h);
  const int b = W.b, bb = b * b;
  std::copy(xs, xs + (size_t)W.nr * b, x);
  std::vector<double> r(b);
  for (int w = 0; w < W.nw; ++w) {
    const int row = W.nr + w;
    for (int k = 0; k < b; ++k) r[k] = g[(size_t)row * b + k];
    for (int p = W.A.rp[row]; p < W.A.rp[row + 1]; ++p) {
      const int c = W.A.ci[p];
      if (c == row) continue;
      const double* awc = &W.A.v[(size_t)p * bb];
      for (int i = 0; i < b; ++i) {
        double acc = 0.0;
        for (int k = 0; k < b; ++k) acc += awc[i * b + k] * xs[(size_t)c * b + k];
        r[i] -= acc;
      }
    }
    const double* wi = &W.winv[(size_t)w * bb];
    for (int i = 0; i < b; ++i) {
      double acc = 0.0;
      for (int k = 0; k < b; ++k) acc += wi[i * b + k] * r[k];
      x[(size_t)row * b + i] = acc;
    }
  }
}

int orc_jp_colouring(int n, const int* rp, const int* ci, int* colour) {
  Csr S = adjacency(n, rp, ci);
  std::vector<int> c;
  const int g = jp_greedy_colouring(S, c);
  std::copy(c.begin(), c.end(), colour);
  return g;
}

int orc_vertices_grouping(int n, const int* rp, const int* ci, int* colour) {
  Csr S = adjacency(n, rp, ci);
  std::vector<int> c;
  int g = vertices_grouping(S, c);
  std::copy(c.begin(), c.end(), colour);
  return g;
}

// Standalone PGS-MC sweep (Algorithm 4.3) on a CSR matrix already in colour order.
int orc_pgs_mc(int n, const int* rp, const int* ci, const double* v, int g, const int* cptr,
               const double* b, double* x, int forward) {
  Csr a;
  a.n = n;
  a.rp.assign(rp, rp + n + 1);
  a.ci.assign(ci, ci + rp[n]);
  a.v.assign(v, v + rp[n]);
  std::vector<int> cp(cptr, cptr + g + 1);
  gs_sweep(a, cp, b, x, forward != 0);
  return ORC_OK;
}

// Standalone pairwise matching pass and Galerkin product (for the aggregation pins).
int orc_pairwise(int n, const int* rp, const int* ci, const double* v, double beta,
                 unsigned long long seed, int* agg) {
  Csr a;
  a.n = n;
  a.rp.assign(rp, rp + n + 1);
  a.ci.assign(ci, ci + rp[n]);
  a.v.assign(v, v + rp[n]);
  std::vector<int> out;
  int nc = pairwise_matching(a, beta, seed, out);
  std::copy(out.begin(), out.end(), agg);
  return nc;
}

unsigned long long orc_splitmix64(unsigned long long x) { return splitmix64(x); }

}  // extern "C"
