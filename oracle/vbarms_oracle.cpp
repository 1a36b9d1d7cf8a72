// VBARMS FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the method of
// "Using the VBARMS method in parallel computing" (Carpentieri, Liao,
// Sosonkina, Bonfiglioli, arXiv 1508.02219), written from the paper.  It is the
// yardstick the CUDA library is checked against.  Only the test suite, the
// smoke check and the benchmark's CPU-baseline leg may load it; the library
// never does.  It shares no code, header or table with the CUDA path.
//
// Every floating-point operation is a separate IEEE round-to-nearest step
// (build with -ffp-contract=off), evaluated in the order written here.
//
// Readings of points the paper leaves open (R1-R9; T1-T3 at compress_two_pass and G1-G5
// at graph_compress; A1-A3 for groups of several supernodes in Step 3; D1-D7 for Section 5):
//  R1  similarity of rows i,j (Section 2.1): cos = |P_i n P_j| / sqrt(|P_i||P_j|)
//      on the stored pattern of the rows; j joins i's group iff cos >= tau,
//      tested exactly as (double)(c*c) >= (tau*tau) * (double)(|P_i||P_j|).
//  R2  greedy in natural order; a row that is still unassigned becomes a
//      leader and claims every unassigned later row similar to the leader.
//  R3  empty rows are singleton groups and similar to nothing.
//  R4  Step 2 scaling: r_i = 1/max_j |a_ij|, then c_j = 1/max_i |r_i a_ij|
//      (zero row/column -> 1); applied at every level.
//  R5  Step 3 weights: w(Y) = ||A_YY||_F / sum_Z ||A_YZ||_F (block-row order),
//      visit by (w desc, index asc), one supernode per independent group.
//  R6  drop rule (Section 3): block B (m x n) is dropped iff
//      ||B||_F^2 < (t*m*n)^2; at most lfil blocks (largest norm, ties to the
//      lower column) are kept per block row of W, G, L_S, U_S when lfil >= 0.
//  R7  the Schur complement is exact except at the last reduction, where the
//      threshold is applied to its off-diagonal blocks.
//  R8  last level: block ILUT in natural order (block IKJ form of Alg. 3).
//  R9  FGMRES(m) with right preconditioning, MGS Arnoldi, Givens rotations,
//      true residual at every restart, stop at ||r|| <= rtol ||b||.
//  D1  Section 5 subdomains on one address space: the compressed block rows
//      are split into N contiguous ranges, part(I) = floor(N * roff_I / n)
//      (the locality-preserving row order stands in for a graph partitioner).
//  D2  overlap: W_i^d = adj(W_i^{d-1}), adj(S) = S plus every block row
//      coupled to S by a stored block of A or A^T; A_i keeps the blocks of A
//      with row and column in W_i^delta, numbered in ascending order.
//  D3  block Jacobi (delta = 0) and additive Schwarz add R_i^T A_i^{-1} R_i
//      over the subdomains in order; the restricted variant keeps from
//      subdomain i only the rows of W_i^0.
//  A1  groups of Step 3 (gs > 1; the diagonal blocks D_i of D block sparse):
//      supernodes visited as in R5; an unmarked eligible one seeds a group,
//      which grows breadth first (members in the order they joined, each
//      member's neighbours in ascending order) by unmarked eligible
//      supernodes until it holds gs of them; then the group's members and
//      all their neighbours are marked.  P_I lists the groups by their
//      smallest member, members ascending, then C ascending.  gs = 1 is R5.
//  A2  the partial factorization with groups splits each pivot the way the
//      single-supernode levels do: sweep 1 over the rows y of [D, F] in
//      order eliminates w_k for the group columns k < y (ascending, fill
//      included) with m = w_k U_k^{-1} (drop test R6), w_j -= m ubar_kj for
//      the blocks j > k of row k (group part and W part); lfil trims the
//      multipliers after use (L); the updated diagonal block is GEPP
//      factored (P_y^T L_y U_y), and the rest of the row becomes
//      ubar_yj = L_y^{-1} P_y w_j (drop test; lfil separately on the group
//      part and on W).  Sweep 2 over the rows of [E, C] eliminates the E
//      part the same way (G candidates; fill only inside a group), keeps
//      the lfil largest as G and forms S = C - G W as for gs = 1.
//  A3  the level solve: u_y = L_y^{-1} P_y (f_y - sum_k m_yk u_k) in order;
//      backward x_y = U_y^{-1} (u_y - W_y z - sum_{j>y} ubar_yj x_j) in
//      reverse order (W terms first, then the group terms ascending).
//  D4  Schur-complement preconditioner (Section 5, eq. paral): on the D1
//      partition (no overlap), block row I is an interface row iff a stored
//      block of A couples it, as row or as column, to a block row of another
//      subdomain; A_i keeps the blocks of A with row and column in subdomain
//      i, interior rows first, then interface rows (each ascending), i.e.
//      [[B_i, F_i], [E_i, C_i]].
//  D5  A_i is factored by VBARMS with the interface rows kept out of every
//      independent set, so they reach the last level, after the remaining
//      interior rows; the trailing interface rows of its block ILUT are
//      L_S U_S, the by-product approximation of S_i = C_i - E_i B_i^{-1} F_i.
//  D6  one application to r = (f_i, g_i): z = the interface parts of the
//      local solves of r_i (= S_i^{-1} g'_i); y from msteps steps of GMRES
//      (y_0 = 0, MGS, Givens, early stop on a zero Arnoldi norm) on
//      (I + S^{-1} E) y = z: eq. gschur preconditioned by blockdiag(S_i),
//      E the couplings E_ij; S_i^{-1} v = the interface part of the local
//      solve of (0, v).
//  D7  eq. loc_var_schur: u_i = the interior part of the local solve of r_i
//      whose last-level backward sweep takes the interface unknowns from y_i
//      (divided by the column scalings of each level on the way down)
//      instead of solving for them; the result is (u_i, y_i).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

namespace {

enum { OK = 0, EINVAL = 1, ESINGULAR = 4, ENOCONV = 6 };

// ---------------------------------------------------------------------------
// Variable block compressed sparse row matrix (VBCSR, Section 2 and 3.1):
// each stored block is a dense row-major rsz[I] x csz[J] array.
struct VB {
  int64_t nbr = 0, nbc = 0;
  std::vector<int32_t> rsz, csz;
  std::vector<int64_t> roff, coff;  // scalar offsets of block rows / cols
  std::vector<int64_t> bptr{0};
  std::vector<int32_t> bcol;
  std::vector<int64_t> voff{0};
  std::vector<double> val;

  void init(const std::vector<int32_t>& r, const std::vector<int32_t>& c) {
    rsz = r;
    csz = c;
    nbr = (int64_t)r.size();
    nbc = (int64_t)c.size();
    roff.assign(nbr + 1, 0);
    coff.assign(nbc + 1, 0);
    for (int64_t i = 0; i < nbr; ++i) roff[i + 1] = roff[i] + rsz[i];
    for (int64_t j = 0; j < nbc; ++j) coff[j + 1] = coff[j] + csz[j];
    bptr.assign(1, 0);
    bcol.clear();
    voff.assign(1, 0);
    val.clear();
  }
  // Append a block to the row being built (rows are built in order).
  void push(int32_t col, const double* data) {
    int64_t row = (int64_t)bptr.size() - 1;
    int64_t sz = (int64_t)rsz[row] * csz[col];
    bcol.push_back(col);
    val.insert(val.end(), data, data + sz);
    voff.push_back((int64_t)val.size());
  }
  void end_row() { bptr.push_back((int64_t)bcol.size()); }
  int64_t nnzb() const { return (int64_t)bcol.size(); }
  double* blk(int64_t b) { return val.data() + voff[b]; }
  const double* blk(int64_t b) const { return val.data() + voff[b]; }
  int64_t find(int64_t row, int32_t col) const {
    for (int64_t b = bptr[row]; b < bptr[row + 1]; ++b)
      if (bcol[b] == col) return b;
    return -1;
  }
};

// Squared Frobenius norm, summed in row-major order.
double fro2(const double* a, int64_t cnt) {
  double s = 0.0;
  for (int64_t e = 0; e < cnt; ++e) s = s + a[e] * a[e];
  return s;
}

// Drop test of Section 3: ||B||_F / (m n) < t, compared squared (R6).
bool dropped(const double* a, int m, int n, double t) {
  double thr = t * (double)m * (double)n;
  return fro2(a, (int64_t)m * n) < thr * thr;
}

// ---------------------------------------------------------------------------
// Gaussian elimination with partial pivoting of one dense m x m pivot block;
// Section 3 states that block pivots are factored exactly this way.  In place: unit-lower L below the
// diagonal, U on and above it; piv[k] = row swapped with row k at step k.
// The pivot is the largest |a_ik|, the lowest row on ties.
int gepp(double* a, int m, int32_t* piv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = std::fabs(a[(int64_t)k * m + k]);
    for (int i = k + 1; i < m; ++i) {
      double v = std::fabs(a[(int64_t)i * m + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (best == 0.0) return ESINGULAR;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < m; ++j) std::swap(a[(int64_t)k * m + j], a[(int64_t)p * m + j]);
    double d = a[(int64_t)k * m + k];
    for (int i = k + 1; i < m; ++i) {
      double l = a[(int64_t)i * m + k] / d;
      a[(int64_t)i * m + k] = l;
      for (int j = k + 1; j < m; ++j)
        a[(int64_t)i * m + j] = a[(int64_t)i * m + j] - l * a[(int64_t)k * m + j];
    }
  }
  return OK;
}

// X (m x n) <- L^{-1} P X for a GEPP-factored m x m block (lu, piv).
void apply_LinvP(const double* lu, const int32_t* piv, int m, double* x, int n) {
  for (int k = 0; k < m; ++k)
    if (piv[k] != k)
      for (int j = 0; j < n; ++j) std::swap(x[(int64_t)k * n + j], x[(int64_t)piv[k] * n + j]);
  for (int i = 1; i < m; ++i)
    for (int k = 0; k < i; ++k) {
      double l = lu[(int64_t)i * m + k];
      for (int j = 0; j < n; ++j) x[(int64_t)i * n + j] = x[(int64_t)i * n + j] - l * x[(int64_t)k * n + j];
    }
}

// X (m x n) <- U^{-1} X (back substitution, column by column).
void apply_Uinv_left(const double* lu, int m, double* x, int n) {
  for (int i = m - 1; i >= 0; --i) {
    for (int j = 0; j < n; ++j) {
      double s = x[(int64_t)i * n + j];
      for (int k = i + 1; k < m; ++k) s = s - lu[(int64_t)i * m + k] * x[(int64_t)k * n + j];
      x[(int64_t)i * n + j] = s / lu[(int64_t)i * m + i];
    }
  }
}

// X (r x m) <- X U^{-1} (row by row, forward over columns).
void apply_Uinv_right(const double* lu, int m, double* x, int r) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < m; ++j) {
      double s = x[(int64_t)i * m + j];
      for (int k = 0; k < j; ++k) s = s - x[(int64_t)i * m + k] * lu[(int64_t)k * m + j];
      x[(int64_t)i * m + j] = s / lu[(int64_t)j * m + j];
    }
}

// X (r x m) <- X (P^T L U)^{-1} = X U^{-1} L^{-1} P.
void apply_Ainv_right(const double* lu, const int32_t* piv, int m, double* x, int r) {
  apply_Uinv_right(lu, m, x, r);
  for (int i = 0; i < r; ++i)
    for (int j = m - 1; j >= 0; --j) {
      double s = x[(int64_t)i * m + j];
      for (int q = j + 1; q < m; ++q) s = s - x[(int64_t)i * m + q] * lu[(int64_t)q * m + j];
      x[(int64_t)i * m + j] = s;
    }
  for (int k = m - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int i = 0; i < r; ++i) std::swap(x[(int64_t)i * m + k], x[(int64_t)i * m + piv[k]]);
}

// B (r x n) <- B - X (r x m) * Y (m x n), each element's terms in k order.
void sub_prod(double* b, const double* x, const double* y, int r, int m, int n) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < n; ++j) {
      double a = b[(int64_t)i * n + j];
      for (int k = 0; k < m; ++k) a = a - x[(int64_t)i * m + k] * y[(int64_t)k * n + j];
      b[(int64_t)i * n + j] = a;
    }
}

// Keep at most lfil of the candidate blocks of one block row: the largest
// squared norms, the lower column on ties (R6).  Returns kept indices in
// ascending column order.
std::vector<int> select_lfil(const std::vector<int32_t>& cols, const std::vector<double>& f2, int lfil) {
  std::vector<int> idx(cols.size());
  std::iota(idx.begin(), idx.end(), 0);
  if (lfil >= 0 && (int64_t)idx.size() > lfil) {
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
      if (f2[a] != f2[b]) return f2[a] > f2[b];
      return cols[a] < cols[b];
    });
    idx.resize(lfil);
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return cols[a] < cols[b]; });
  return idx;
}

// ---------------------------------------------------------------------------
// Step 1: angle-based compression (Section 2.1) and the block permutation
// P_B A P_B^T of Eq. 3, stored as VBCSR.
struct Compressed {
  VB A;
  std::vector<int32_t> perm;  // perm[k] = original row at permuted position k
  std::vector<int32_t> bsz;
  double av_bd = 0, av_bs = 0;
};

bool csr_ok(int64_t n, const int64_t* rowptr, const int32_t* colind) {
  if (n < 0) return false;
  if (n > 0 && rowptr[0] != 0) return false;
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return false;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (colind[p] < 0 || colind[p] >= n) return false;
      if (p > rowptr[i] && colind[p] <= colind[p - 1]) return false;
    }
  }
  return true;
}

void assemble(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
              const std::vector<std::vector<int32_t>>& members, Compressed& out);

int compress(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau,
             Compressed& out) {
  if (!(tau > 0.0 && tau <= 1.0) || !csr_ok(n, rowptr, colind)) return EINVAL;
  // Column lists of the pattern matrix C (rows having a stored entry in col c).
  std::vector<int64_t> cptr(n + 1, 0);
  for (int64_t p = 0; p < (n ? rowptr[n] : 0); ++p) cptr[colind[p] + 1]++;
  for (int64_t c = 0; c < n; ++c) cptr[c + 1] += cptr[c];
  std::vector<int32_t> crow(n ? rowptr[n] : 0);
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - (n ? 1 : 0));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) crow[fill[colind[p]]++] = (int32_t)i;
  }
  // Greedy grouping (R1-R3): (C C^T)_{ij} = |P_i n P_j| for the leader i.
  const double tau2 = tau * tau;
  std::vector<int64_t> leader(n, -1);
  std::vector<int32_t> cnt(n, 0);
  std::vector<int64_t> touched;
  for (int64_t i = 0; i < n; ++i) {
    if (leader[i] != -1) continue;
    leader[i] = i;
    const int64_t ni = rowptr[i + 1] - rowptr[i];
    if (ni == 0) continue;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int32_t c = colind[p];
      for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
        int64_t j = crow[q];
        if (j > i && leader[j] == -1 && cnt[j]++ == 0) touched.push_back(j);
      }
    }
    for (int64_t j : touched) {
      const int64_t c = cnt[j];
      const int64_t nj = rowptr[j + 1] - rowptr[j];
      if ((double)(c * c) >= tau2 * (double)(ni * nj)) leader[j] = i;
      cnt[j] = 0;
    }
    touched.clear();
  }
  // Blocks in leader order, members ascending.
  std::vector<int32_t> blk_of_leader(n, -1);
  int32_t p = 0;
  for (int64_t i = 0; i < n; ++i)
    if (leader[i] == i) blk_of_leader[i] = p++;
  std::vector<std::vector<int32_t>> members(p);
  for (int64_t i = 0; i < n; ++i) members[blk_of_leader[leader[i]]].push_back((int32_t)i);
  assemble(n, rowptr, colind, val, members, out);
  return OK;
}

// The block permutation of the given groups (in the given order, members in
// the given order) and the VBCSR of P_B A P_B^T, with av_bd and av_bs.
void assemble(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
              const std::vector<std::vector<int32_t>>& members, Compressed& out) {
  const int32_t p = (int32_t)members.size();
  out.perm.clear();
  out.bsz.assign(p, 0);
  std::vector<int32_t> blk(n), off(n);
  for (int32_t b = 0; b < p; ++b) {
    out.bsz[b] = (int32_t)members[b].size();
    for (size_t k = 0; k < members[b].size(); ++k) {
      blk[members[b][k]] = b;
      off[members[b][k]] = (int32_t)k;
      out.perm.push_back(members[b][k]);
    }
  }
  // VBCSR of P_B A P_B^T: block (I,J) is stored iff a stored entry of A falls
  // in it; blocks are zero padded and values copied unchanged.
  out.A.init(out.bsz, out.bsz);
  int64_t pos = 0;
  double padded = 0.0;
  for (int32_t I = 0; I < p; ++I) {
    std::vector<int32_t> cols;
    for (int32_t r : members[I])
      for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) cols.push_back(blk[colind[q]]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    std::vector<std::vector<double>> data(cols.size());
    for (size_t t = 0; t < cols.size(); ++t) data[t].assign((size_t)out.bsz[I] * out.bsz[cols[t]], 0.0);
    for (int32_t r : members[I])
      for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        int32_t J = blk[colind[q]];
        size_t t = std::lower_bound(cols.begin(), cols.end(), J) - cols.begin();
        data[t][(size_t)off[r] * out.bsz[J] + off[colind[q]]] = val[q];
      }
    for (size_t t = 0; t < cols.size(); ++t) {
      out.A.push(cols[t], data[t].data());
      padded += (double)data[t].size();
    }
    out.A.end_row();
    pos += out.bsz[I];
  }
  (void)pos;
  const double nnz = n ? (double)rowptr[n] : 0.0;
  out.av_bd = padded > 0 ? nnz / padded : 0.0;
  out.av_bs = p > 0 ? (double)n / (double)p : 0.0;
}

// ---------------------------------------------------------------------------
// Two-pass variant of the angle method (Section 2.1), readings T1-T3:
//  T1 pass 1 groups rows with identical stored patterns P_i (the rows of the
//     pattern matrix); a class of two or more rows is a group, the rows of
//     one-row classes are unassigned.
//  T2 pass 2 takes the unassigned rows in natural order; each joins the first
//     group (groups in ascending order of their smallest row) whose common
//     pattern P_g passes the angle test of R1 against P_j; the groups keep
//     their pattern; a row that fits no group (and an empty row) stays alone.
//  T3 blocks in ascending order of their smallest row, rows ascending.
int compress_two_pass(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau,
                      Compressed& out) {
  if (!(tau > 0.0 && tau <= 1.0) || !csr_ok(n, rowptr, colind)) return EINVAL;
  // T1: classes of identical patterns (rows compared after sorting by pattern)
  std::vector<int32_t> rows(n);
  std::iota(rows.begin(), rows.end(), 0);
  auto pat_less = [&](int32_t a, int32_t b) {
    return std::lexicographical_compare(colind + rowptr[a], colind + rowptr[a + 1], colind + rowptr[b],
                                        colind + rowptr[b + 1]);
  };
  auto pat_eq = [&](int32_t a, int32_t b) {
    return rowptr[a + 1] - rowptr[a] == rowptr[b + 1] - rowptr[b] &&
           std::equal(colind + rowptr[a], colind + rowptr[a + 1], colind + rowptr[b]);
  };
  std::stable_sort(rows.begin(), rows.end(), pat_less);
  std::vector<std::vector<int32_t>> groups;  // pass-1 groups (two or more rows)
  std::vector<char> assigned(n, 0);
  for (int64_t a = 0; a < n;) {
    int64_t b = a + 1;
    while (b < n && pat_eq(rows[a], rows[b])) ++b;
    if (b - a >= 2 && rowptr[rows[a] + 1] > rowptr[rows[a]]) {
      std::vector<int32_t> g(rows.begin() + a, rows.begin() + b);
      std::sort(g.begin(), g.end());
      for (int32_t r : g) assigned[r] = 1;
      groups.push_back(std::move(g));
    }
    a = b;
  }
  std::sort(groups.begin(), groups.end(),
            [](const std::vector<int32_t>& x, const std::vector<int32_t>& y) { return x[0] < y[0]; });
  const size_t ng = groups.size();
  std::vector<int32_t> ref(ng);  // a row carrying each group's pattern
  for (size_t g = 0; g < ng; ++g) ref[g] = groups[g][0];
  // T2: unassigned rows against the groups, R1's exact test
  const double tau2 = tau * tau;
  std::vector<std::vector<int32_t>> joined(ng);
  std::vector<std::vector<int32_t>> members;
  std::vector<char> mark(n, 0);
  for (int64_t j = 0; j < n; ++j) {
    if (assigned[j]) continue;
    const int64_t nj = rowptr[j + 1] - rowptr[j];
    int64_t hit = -1;
    if (nj > 0) {
      for (int64_t q = rowptr[j]; q < rowptr[j + 1]; ++q) mark[colind[q]] = 1;
      for (size_t g = 0; g < ng && hit < 0; ++g) {
        const int32_t r = ref[g];
        const int64_t nr = rowptr[r + 1] - rowptr[r];
        int64_t c = 0;
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) c += mark[colind[q]];
        if ((double)(c * c) >= tau2 * (double)(nj * nr)) hit = (int64_t)g;
      }
      for (int64_t q = rowptr[j]; q < rowptr[j + 1]; ++q) mark[colind[q]] = 0;
    }
    if (hit >= 0)
      joined[hit].push_back((int32_t)j);
    else
      members.push_back({(int32_t)j});
  }
  for (size_t g = 0; g < ng; ++g) {
    std::vector<int32_t> m;
    std::merge(groups[g].begin(), groups[g].end(), joined[g].begin(), joined[g].end(), std::back_inserter(m));
    members.push_back(std::move(m));
  }
  // T3
  std::sort(members.begin(), members.end(),
            [](const std::vector<int32_t>& x, const std::vector<int32_t>& y) { return x[0] < y[0]; });
  assemble(n, rowptr, colind, val, members, out);
  return OK;
}

// ---------------------------------------------------------------------------
// Graph-based compression (Section 2.2, Alg. 1), readings G1-G5:
//  G1 adj(i) is the closed neighbourhood of i in the graph of A + A^T
//     ({i} plus every j with a stored a_ij or a_ji); the key of i is
//     chk(i) = sum of adj(i).
//  G2 supernodes: vertices scanned by (key, index); the first unassigned
//     vertex of a key opens a supernode and takes every later vertex of the
//     same key with an identical adj (so a supernode's first vertex is its
//     smallest).
//  G3 merge phase: supernodes visited in ascending order of their smallest
//     vertex; X's candidates are the supernodes (as they are when X's turn
//     starts) whose adjacency meets X, i.e. the owners of adj(X), X excluded,
//     in ascending order of their smallest vertex, each tried once.
//  G4 X and Z merge iff the density of the merged supernode's block row and
//     column, N / T with T and N of Section 2.2, is at least mu, tested as
//     (double)N >= mu * (double)T.
//  G5 blocks in ascending order of their smallest vertex, vertices ascending.
struct GNode {
  std::vector<int32_t> v;    // vertices, ascending
  std::vector<int32_t> adj;  // union of adj(v), ascending
  int64_t deg = 0;           // sum of |adj(v)|
  int64_t inner = 0;         // sum of |adj(v) n X|
  bool alive = true;
};

// T and N of a vertex set S with union adjacency a, degree sum deg and inner
// count inner (Section 2.2): rows and columns spanned, nonzeros spanned.
inline int64_t span_T(int64_t s, int64_t a) { return 2 * a * s - s * s; }
inline int64_t span_N(int64_t deg, int64_t inner) { return 2 * deg - inner; }

int graph_compress(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double mu,
                   Compressed& out) {
  if (!(mu >= 0.0) || !csr_ok(n, rowptr, colind)) return EINVAL;
  // G1: closed neighbourhoods in A + A^T
  std::vector<std::vector<int32_t>> adj(n);
  for (int64_t i = 0; i < n; ++i) {
    adj[i].push_back((int32_t)i);
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      adj[i].push_back(colind[q]);
      adj[colind[q]].push_back((int32_t)i);
    }
  }
  std::vector<int64_t> key(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
    for (int32_t j : adj[i]) key[i] += j;
  }
  // G2: the checksum scan
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::vector<char> done(n, 0);
  std::vector<GNode> V;
  for (int64_t x = 0; x < n; ++x) {
    const int32_t i = order[x];
    if (done[i]) continue;
    GNode Y;
    Y.v.push_back(i);
    done[i] = 1;
    for (int64_t y = x + 1; y < n && key[order[y]] == key[i]; ++y) {
      const int32_t j = order[y];
      if (!done[j] && adj[j] == adj[i]) {
        Y.v.push_back(j);
        done[j] = 1;
      }
    }
    V.push_back(std::move(Y));
  }
  // G3: supernodes by their smallest vertex
  std::sort(V.begin(), V.end(), [](const GNode& a, const GNode& b) { return a.v[0] < b.v[0]; });
  std::vector<int32_t> owner(n);
  for (size_t z = 0; z < V.size(); ++z) {
    GNode& Z = V[z];
    std::sort(Z.v.begin(), Z.v.end());
    for (int32_t v : Z.v) owner[v] = (int32_t)z;
    Z.adj = adj[Z.v[0]];  // identical for every vertex of Z
    for (int32_t v : Z.v) Z.deg += (int64_t)adj[v].size();
  }
  for (size_t z = 0; z < V.size(); ++z) {
    V[z].inner = 0;
    for (int32_t v : V[z].v)
      for (int32_t u : adj[v]) V[z].inner += owner[u] == (int32_t)z ? 1 : 0;
  }
  for (size_t x = 0; x < V.size(); ++x) {
    if (!V[x].alive) continue;
    std::vector<int32_t> cand;
    for (int32_t u : V[x].adj)
      if (owner[u] != (int32_t)x) cand.push_back(owner[u]);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) { return V[a].v[0] < V[b].v[0]; });
    for (int32_t z : cand) {
      GNode& X = V[x];
      GNode& Z = V[z];
      std::vector<int32_t> un;
      std::set_union(X.adj.begin(), X.adj.end(), Z.adj.begin(), Z.adj.end(), std::back_inserter(un));
      int64_t cross = 0;  // sum over v in Z of |adj(v) n X|
      for (int32_t v : Z.v)
        for (int32_t u : adj[v]) cross += owner[u] == (int32_t)x ? 1 : 0;
      const int64_t sz = (int64_t)(X.v.size() + Z.v.size());
      const int64_t T = span_T(sz, (int64_t)un.size());
      const int64_t N = span_N(X.deg + Z.deg, X.inner + Z.inner + 2 * cross);
      if ((double)N >= mu * (double)T) {
        for (int32_t v : Z.v) owner[v] = (int32_t)x;
        std::vector<int32_t> mv;
        std::merge(X.v.begin(), X.v.end(), Z.v.begin(), Z.v.end(), std::back_inserter(mv));
        X.v.swap(mv);
        X.adj.swap(un);
        X.deg += Z.deg;
        X.inner += Z.inner + 2 * cross;
        Z.alive = false;
      }
    }
  }
  // G5
  std::vector<std::vector<int32_t>> members;
  for (auto& X : V)
    if (X.alive) members.push_back(X.v);
  std::sort(members.begin(), members.end(),
            [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) { return a[0] < b[0]; });
  assemble(n, rowptr, colind, val, members, out);
  return OK;
}

// ---------------------------------------------------------------------------
// Step 2 (R4): two-sided max-abs scaling, in place; returns r, c.
void scale(VB& A, std::vector<double>& r, std::vector<double>& c) {
  const int64_t n = A.roff[A.nbr];
  std::vector<double> rmax(n, 0.0), cmax(A.coff[A.nbc], 0.0);
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      const int m = A.rsz[I], nc = A.csz[A.bcol[b]];
      const double* a = A.blk(b);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < nc; ++j) rmax[A.roff[I] + i] = std::max(rmax[A.roff[I] + i], std::fabs(a[i * nc + j]));
    }
  r.assign(n, 1.0);
  for (int64_t i = 0; i < n; ++i)
    if (rmax[i] > 0.0) r[i] = 1.0 / rmax[i];
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      const int m = A.rsz[I], nc = A.csz[A.bcol[b]];
      const int64_t c0 = A.coff[A.bcol[b]];
      const double* a = A.blk(b);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < nc; ++j)
          cmax[c0 + j] = std::max(cmax[c0 + j], std::fabs(r[A.roff[I] + i] * a[i * nc + j]));
    }
  c.assign(A.coff[A.nbc], 1.0);
  for (int64_t j = 0; j < (int64_t)c.size(); ++j)
    if (cmax[j] > 0.0) c[j] = 1.0 / cmax[j];
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      const int m = A.rsz[I], nc = A.csz[A.bcol[b]];
      const int64_t c0 = A.coff[A.bcol[b]];
      double* a = A.blk(b);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < nc; ++j) a[i * nc + j] = (r[A.roff[I] + i] * a[i * nc + j]) * c[c0 + j];
    }
}

// ---------------------------------------------------------------------------
// Step 3 (R5): weighted greedy block independent set on the quotient graph of
// A + A^T (Section 3, edge set E_B), self loops removed.  Returns pI (D
// supernodes ascending, then C supernodes ascending) and the D count.
// fixed (optional): rows that never enter the set (D5).
void is_order(const VB& A, double ddtol, std::vector<int32_t>& pI, int64_t& nD, std::vector<double>& w,
              const std::vector<char>* fixed = nullptr) {
  const int64_t p = A.nbr;
  w.assign(p, 0.0);
  for (int64_t Y = 0; Y < p; ++Y) {
    double dsum = 0.0, diag = 0.0;
    for (int64_t b = A.bptr[Y]; b < A.bptr[Y + 1]; ++b) {
      double f = std::sqrt(fro2(A.blk(b), (int64_t)A.rsz[Y] * A.csz[A.bcol[b]]));
      dsum = dsum + f;
      if (A.bcol[b] == Y) diag = f;
    }
    w[Y] = dsum > 0.0 ? diag / dsum : 0.0;
  }
  std::vector<std::vector<int32_t>> adj(p);
  for (int64_t Y = 0; Y < p; ++Y)
    for (int64_t b = A.bptr[Y]; b < A.bptr[Y + 1]; ++b) {
      int32_t Z = A.bcol[b];
      if (Z == Y) continue;
      adj[Y].push_back(Z);
      adj[Z].push_back((int32_t)Y);
    }
  std::vector<int32_t> order(p);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (w[a] != w[b]) return w[a] > w[b];
    return a < b;
  });
  std::vector<char> marked(p, 0), inD(p, 0);
  for (int32_t v : order) {
    if (marked[v]) continue;
    if (w[v] < ddtol) continue;
    if (fixed && (*fixed)[v]) continue;
    inD[v] = 1;
    marked[v] = 1;
    for (int32_t u : adj[v]) marked[u] = 1;
  }
  pI.clear();
  for (int64_t Y = 0; Y < p; ++Y)
    if (inD[Y]) pI.push_back((int32_t)Y);
  nD = (int64_t)pI.size();
  for (int64_t Y = 0; Y < p; ++Y)
    if (!inD[Y]) pI.push_back((int32_t)Y);
}

// Step 3 with groups (A1): up to gs supernodes per independent group.  gptr
// returns the group boundaries over the D positions of pI.
void is_order_groups(const VB& A, double ddtol, int gs, std::vector<int32_t>& pI, int64_t& nD,
                     std::vector<double>& w, std::vector<int64_t>& gptr, const std::vector<char>* fixed) {
  const int64_t p = A.nbr;
  std::vector<int32_t> pI1;
  int64_t nD1 = 0;
  is_order(A, ddtol, pI1, nD1, w, fixed);  // the weights (R5)
  std::vector<std::vector<int32_t>> adj(p);
  for (int64_t Y = 0; Y < p; ++Y)
    for (int64_t b = A.bptr[Y]; b < A.bptr[Y + 1]; ++b) {
      const int32_t Z = A.bcol[b];
      if (Z == Y) continue;
      adj[Y].push_back(Z);
      adj[Z].push_back((int32_t)Y);
    }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  std::vector<int32_t> order(p);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (w[a] != w[b]) return w[a] > w[b];
    return a < b;
  });
  auto eligible = [&](int32_t v) { return !(w[v] < ddtol) && !(fixed && (*fixed)[v]); };
  std::vector<char> marked(p, 0);
  std::vector<std::vector<int32_t>> groups;
  for (int32_t v : order) {
    if (marked[v] || !eligible(v)) continue;
    std::vector<int32_t> grp{v};
    marked[v] = 1;
    for (size_t head = 0; head < grp.size() && (int)grp.size() < gs; ++head)
      for (int32_t z : adj[grp[head]]) {
        if ((int)grp.size() >= gs) break;
        if (marked[z] || !eligible(z)) continue;
        grp.push_back(z);
        marked[z] = 1;
      }
    for (int32_t u : grp)
      for (int32_t z : adj[u]) marked[z] = 1;
    std::sort(grp.begin(), grp.end());
    groups.push_back(std::move(grp));
  }
  std::sort(groups.begin(), groups.end(),
            [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) { return a[0] < b[0]; });
  std::vector<char> inD(p, 0);
  pI.clear();
  gptr.assign(1, 0);
  for (auto& g : groups) {
    for (int32_t v : g) {
      pI.push_back(v);
      inD[v] = 1;
    }
    gptr.push_back((int64_t)pI.size());
  }
  nD = (int64_t)pI.size();
  for (int64_t Y = 0; Y < p; ++Y)
    if (!inD[Y]) pI.push_back((int32_t)Y);
}

// ---------------------------------------------------------------------------
struct Level {
  VB A;  // input of the level after Step 2 scaling
  std::vector<double> r, c, w;
  std::vector<int32_t> pI;
  int64_t nD = 0, nC = 0;
  VB D;  // pivot blocks (block diagonal), LU in place
  std::vector<int32_t> piv;
  VB F, E, C, W, G, S;
  bool grouped = false;       // A2: D block sparse within groups
  std::vector<int64_t> gptr;  // group boundaries over the D rows
  VB Lg, Ug;                  // group multipliers (below) and group part of Ubar (above the diagonal)
};

struct Last {
  VB A;  // scaled last-level matrix
  std::vector<double> r, c;
  VB Dg;  // pivot blocks, LU in place
  std::vector<int32_t> piv;
  VB L, U;
};

struct Prec {
  std::vector<Level> lev;
  Last last;
  std::vector<char> last_fixed;  // D5: the fixed rows at the last level (empty: none)
  int64_t n = 0;
  double fill = 0;  // stored scalars of all factors
};

// Steps 3-4 for one level (Eq. 4-6) in the two-sweep form of Section 3.1.
int factor_level(Level& L, bool last_reduction, double t, int lfil) {
  const VB& A = L.A;
  const int64_t p = A.nbr;
  std::vector<int32_t> newpos(p);
  for (int64_t k = 0; k < p; ++k) newpos[L.pI[k]] = (int32_t)k;
  L.nC = p - L.nD;
  std::vector<int32_t> szD(L.nD), szC(L.nC);
  for (int64_t k = 0; k < p; ++k) (k < L.nD ? szD[k] : szC[k - L.nD]) = A.rsz[L.pI[k]];
  // P_I (S1 A S2) P_I^T = [[D, F], [E, C]]  (Eq. 4).
  L.D.init(szD, szD);
  L.F.init(szD, szC);
  L.E.init(szC, szD);
  L.C.init(szC, szC);
  std::vector<double> zero;
  for (int64_t k = 0; k < p; ++k) {
    const int32_t Y = L.pI[k];
    const bool rowD = k < L.nD;
    bool has_diag = false;
    for (int64_t b = A.bptr[Y]; b < A.bptr[Y + 1]; ++b) {
      const int32_t nz = newpos[A.bcol[b]];
      const bool colD = nz < L.nD;
      if (rowD) {
        if (colD) {
          // Only the diagonal block: D supernodes are pairwise uncoupled.
          L.D.push((int32_t)k, A.blk(b));
          has_diag = true;
        } else {
          L.F.push((int32_t)(nz - L.nD), A.blk(b));
        }
      } else {
        if (colD)
          L.E.push(nz, A.blk(b));
        else
          L.C.push((int32_t)(nz - L.nD), A.blk(b));
      }
    }
    if (rowD) {
      if (!has_diag) return ESINGULAR;  // zero pivot block
      L.D.end_row();
      L.F.end_row();
    } else {
      L.E.end_row();
      L.C.end_row();
    }
  }
  // Sweep 1 over the block rows [D, F]: D_y = P_y^T L_y U_y and
  // W = L^{-1} P F (the block row [U, L^{-1} F] of Eq. 5), with dropping.
  L.piv.assign(L.D.roff[L.nD], 0);
  for (int64_t y = 0; y < L.nD; ++y) {
    if (gepp(L.D.blk(L.D.bptr[y]), szD[y], L.piv.data() + L.D.roff[y]) != OK) return ESINGULAR;
  }
  L.W.init(szD, szC);
  for (int64_t y = 0; y < L.nD; ++y) {
    const int m = szD[y];
    std::vector<int32_t> cols;
    std::vector<double> f2;
    std::vector<std::vector<double>> blocks;
    for (int64_t b = L.F.bptr[y]; b < L.F.bptr[y + 1]; ++b) {
      const int ns = szC[L.F.bcol[b]];
      std::vector<double> x(L.F.blk(b), L.F.blk(b) + (int64_t)m * ns);
      apply_LinvP(L.D.blk(L.D.bptr[y]), L.piv.data() + L.D.roff[y], m, x.data(), ns);
      if (dropped(x.data(), m, ns, t)) continue;
      cols.push_back(L.F.bcol[b]);
      f2.push_back(fro2(x.data(), (int64_t)m * ns));
      blocks.push_back(std::move(x));
    }
    for (int k : select_lfil(cols, f2, lfil)) L.W.push(cols[k], blocks[k].data());
    L.W.end_row();
  }
  // Sweep 2 over the block rows [E, C]: multipliers G = E U^{-1} and the
  // Schur complement S = C - G W = C - E D^{-1} F (Eq. 6).
  L.G.init(szC, szD);
  L.S.init(szC, szC);
  for (int64_t r = 0; r < L.nC; ++r) {
    const int nr = szC[r];
    std::vector<int32_t> cols;
    std::vector<double> f2;
    std::vector<std::vector<double>> blocks;
    for (int64_t b = L.E.bptr[r]; b < L.E.bptr[r + 1]; ++b) {
      const int32_t y = L.E.bcol[b];
      const int m = szD[y];
      std::vector<double> x(L.E.blk(b), L.E.blk(b) + (int64_t)nr * m);
      apply_Uinv_right(L.D.blk(L.D.bptr[y]), m, x.data(), nr);
      if (dropped(x.data(), nr, m, t)) continue;
      cols.push_back(y);
      f2.push_back(fro2(x.data(), (int64_t)nr * m));
      blocks.push_back(std::move(x));
    }
    std::vector<int> keep = select_lfil(cols, f2, lfil);
    for (int k : keep) L.G.push(cols[k], blocks[k].data());
    L.G.end_row();
    std::map<int32_t, std::vector<double>> acc;
    for (int64_t b = L.C.bptr[r]; b < L.C.bptr[r + 1]; ++b)
      acc[L.C.bcol[b]].assign(L.C.blk(b), L.C.blk(b) + (int64_t)nr * szC[L.C.bcol[b]]);
    for (int k : keep) {
      const int32_t y = cols[k];
      const int m = szD[y];
      for (int64_t b = L.W.bptr[y]; b < L.W.bptr[y + 1]; ++b) {
        const int32_t s = L.W.bcol[b];
        std::vector<double>& blk = acc[s];
        if (blk.empty()) blk.assign((size_t)nr * szC[s], 0.0);
        sub_prod(blk.data(), blocks[k].data(), L.W.blk(b), nr, m, szC[s]);
      }
    }
    for (auto& kv : acc) {
      if (last_reduction && kv.first != r && dropped(kv.second.data(), nr, szC[kv.first], t)) continue;
      L.S.push(kv.first, kv.second.data());
    }
    L.S.end_row();
  }
  return OK;
}

// Steps 3-4 with groups (A2): D block sparse inside groups, the two sweeps
// of Section 3.1 with block IKJ elimination inside each group.
int factor_level_groups(Level& L, bool last_reduction, double t, int lfil) {
  const VB& A = L.A;
  const int64_t p = A.nbr;
  L.grouped = true;
  std::vector<int32_t> newpos(p);
  for (int64_t k = 0; k < p; ++k) newpos[L.pI[k]] = (int32_t)k;
  L.nC = p - L.nD;
  std::vector<int32_t> szD(L.nD), szC(L.nC);
  for (int64_t k = 0; k < p; ++k) (k < L.nD ? szD[k] : szC[k - L.nD]) = A.rsz[L.pI[k]];
  L.D.init(szD, szD);
  L.F.init(szD, szC);
  L.E.init(szC, szD);
  L.C.init(szC, szC);
  for (int64_t k = 0; k < p; ++k) {
    const int32_t Y = L.pI[k];
    const bool rowD = k < L.nD;
    // columns in the new order (a group's members are ascending and
    // contiguous, so D columns stay sorted; C columns are ascending)
    std::vector<std::pair<int32_t, int64_t>> cols;
    for (int64_t b = A.bptr[Y]; b < A.bptr[Y + 1]; ++b) cols.push_back({newpos[A.bcol[b]], b});
    std::sort(cols.begin(), cols.end());
    for (auto& cb : cols) {
      const int32_t nz = cb.first;
      const bool colD = nz < L.nD;
      if (rowD)
        (colD ? L.D : L.F).push(colD ? nz : (int32_t)(nz - L.nD), A.blk(cb.second));
      else
        (colD ? L.E : L.C).push(colD ? nz : (int32_t)(nz - L.nD), A.blk(cb.second));
    }
    if (rowD) {
      L.D.end_row();
      L.F.end_row();
    } else {
      L.E.end_row();
      L.C.end_row();
    }
  }
  // pivot block of each D row after its elimination, GEPP LU in place
  VB Dp;
  Dp.init(szD, szD);
  L.piv.assign(L.D.roff[L.nD], 0);
  L.Lg.init(szD, szD);
  L.Ug.init(szD, szD);
  L.W.init(szD, szC);
  // sweep 1 over the rows of [D, F]; keys: D columns, then nD + F column
  for (int64_t y = 0; y < L.nD; ++y) {
    const int ny = szD[y];
    auto csize = [&](int64_t key) { return key < L.nD ? szD[key] : szC[key - L.nD]; };
    std::map<int64_t, std::vector<double>> w;
    for (int64_t b = L.D.bptr[y]; b < L.D.bptr[y + 1]; ++b)
      w[L.D.bcol[b]].assign(L.D.blk(b), L.D.blk(b) + (int64_t)ny * szD[L.D.bcol[b]]);
    for (int64_t b = L.F.bptr[y]; b < L.F.bptr[y + 1]; ++b)
      w[L.nD + L.F.bcol[b]].assign(L.F.blk(b), L.F.blk(b) + (int64_t)ny * szC[L.F.bcol[b]]);
    std::vector<int32_t> lcols;
    std::vector<double> lf2;
    std::vector<std::vector<double>> lblocks;
    auto it = w.begin();
    while (it != w.end() && it->first < y) {
      const int32_t k = (int32_t)it->first;
      const int nk = szD[k];
      std::vector<double> m = std::move(it->second);
      w.erase(it);
      apply_Uinv_right(Dp.blk(Dp.bptr[k]), nk, m.data(), ny);
      if (!dropped(m.data(), ny, nk, t)) {
        for (int64_t b = L.Ug.bptr[k]; b < L.Ug.bptr[k + 1]; ++b) {
          const int32_t j = L.Ug.bcol[b];
          std::vector<double>& blk = w[j];
          if (blk.empty()) blk.assign((size_t)ny * szD[j], 0.0);
          sub_prod(blk.data(), m.data(), L.Ug.blk(b), ny, nk, szD[j]);
        }
        for (int64_t b = L.W.bptr[k]; b < L.W.bptr[k + 1]; ++b) {
          const int32_t c = L.W.bcol[b];
          std::vector<double>& blk = w[L.nD + c];
          if (blk.empty()) blk.assign((size_t)ny * szC[c], 0.0);
          sub_prod(blk.data(), m.data(), L.W.blk(b), ny, nk, szC[c]);
        }
        lcols.push_back(k);
        lf2.push_back(fro2(m.data(), (int64_t)ny * nk));
        lblocks.push_back(std::move(m));
      }
      it = w.upper_bound(k);
    }
    for (int k : select_lfil(lcols, lf2, lfil)) L.Lg.push(lcols[k], lblocks[k].data());
    L.Lg.end_row();
    auto d = w.find(y);
    if (d == w.end()) return ESINGULAR;  // zero pivot block
    std::vector<double> dg = d->second;
    int32_t* pv = L.piv.data() + L.D.roff[y];
    if (gepp(dg.data(), ny, pv) != OK) return ESINGULAR;
    Dp.push((int32_t)y, dg.data());
    Dp.end_row();
    std::vector<int32_t> ucols, fcols;
    std::vector<double> uf2, ff2;
    std::vector<std::vector<double>> ublocks, fblocks;
    for (auto& kv : w) {
      if (kv.first <= y) continue;
      const int ns = csize(kv.first);
      std::vector<double> x = kv.second;
      apply_LinvP(dg.data(), pv, ny, x.data(), ns);
      if (dropped(x.data(), ny, ns, t)) continue;
      if (kv.first < L.nD) {
        ucols.push_back((int32_t)kv.first);
        uf2.push_back(fro2(x.data(), (int64_t)ny * ns));
        ublocks.push_back(std::move(x));
      } else {
        fcols.push_back((int32_t)(kv.first - L.nD));
        ff2.push_back(fro2(x.data(), (int64_t)ny * ns));
        fblocks.push_back(std::move(x));
      }
    }
    for (int k : select_lfil(ucols, uf2, lfil)) L.Ug.push(ucols[k], ublocks[k].data());
    L.Ug.end_row();
    for (int k : select_lfil(fcols, ff2, lfil)) L.W.push(fcols[k], fblocks[k].data());
    L.W.end_row();
  }
  L.D = std::move(Dp);
  // sweep 2 over the rows of [E, C]: G = E Ubar^{-1} and S = C - G W
  L.G.init(szC, szD);
  L.S.init(szC, szC);
  for (int64_t r = 0; r < L.nC; ++r) {
    const int nr = szC[r];
    std::map<int32_t, std::vector<double>> e;
    for (int64_t b = L.E.bptr[r]; b < L.E.bptr[r + 1]; ++b)
      e[L.E.bcol[b]].assign(L.E.blk(b), L.E.blk(b) + (int64_t)nr * szD[L.E.bcol[b]]);
    std::vector<int32_t> cols;
    std::vector<double> f2;
    std::vector<std::vector<double>> blocks;
    while (!e.empty()) {
      auto it = e.begin();
      const int32_t k = it->first;
      const int nk = szD[k];
      std::vector<double> m = std::move(it->second);
      e.erase(it);
      apply_Uinv_right(L.D.blk(L.D.bptr[k]), nk, m.data(), nr);
      if (dropped(m.data(), nr, nk, t)) continue;
      for (int64_t b = L.Ug.bptr[k]; b < L.Ug.bptr[k + 1]; ++b) {
        const int32_t j = L.Ug.bcol[b];
        std::vector<double>& blk = e[j];
        if (blk.empty()) blk.assign((size_t)nr * szD[j], 0.0);
        sub_prod(blk.data(), m.data(), L.Ug.blk(b), nr, nk, szD[j]);
      }
      cols.push_back(k);
      f2.push_back(fro2(m.data(), (int64_t)nr * nk));
      blocks.push_back(std::move(m));
    }
    std::vector<int> keep = select_lfil(cols, f2, lfil);
    for (int k : keep) L.G.push(cols[k], blocks[k].data());
    L.G.end_row();
    std::map<int32_t, std::vector<double>> acc;
    for (int64_t b = L.C.bptr[r]; b < L.C.bptr[r + 1]; ++b)
      acc[L.C.bcol[b]].assign(L.C.blk(b), L.C.blk(b) + (int64_t)nr * szC[L.C.bcol[b]]);
    for (int k : keep) {
      const int32_t y = cols[k];
      const int m = szD[y];
      for (int64_t b = L.W.bptr[y]; b < L.W.bptr[y + 1]; ++b) {
        const int32_t sc = L.W.bcol[b];
        std::vector<double>& blk = acc[sc];
        if (blk.empty()) blk.assign((size_t)nr * szC[sc], 0.0);
        sub_prod(blk.data(), blocks[k].data(), L.W.blk(b), nr, m, szC[sc]);
      }
    }
    for (auto& kv : acc) {
      if (last_reduction && kv.first != r && dropped(kv.second.data(), nr, szC[kv.first], t)) continue;
      L.S.push(kv.first, kv.second.data());
    }
    L.S.end_row();
  }
  return OK;
}

// Last level (R8): block ILUT in natural order, the block IKJ form of Alg. 3
// with the dropping of Section 3.
int ilut_last(Last& X, double t, int lfil) {
  const VB& A = X.A;
  const int64_t p = A.nbr;
  X.Dg.init(A.rsz, A.rsz);
  X.L.init(A.rsz, A.rsz);
  X.U.init(A.rsz, A.rsz);
  X.piv.assign(A.roff[p], 0);
  for (int64_t i = 0; i < p; ++i) {
    const int ni = A.rsz[i];
    std::map<int32_t, std::vector<double>> w;
    for (int64_t b = A.bptr[i]; b < A.bptr[i + 1]; ++b)
      w[A.bcol[b]].assign(A.blk(b), A.blk(b) + (int64_t)ni * A.csz[A.bcol[b]]);
    std::vector<int32_t> lcols;
    std::vector<double> lf2;
    std::vector<std::vector<double>> lblocks;
    auto it = w.begin();
    while (it != w.end() && it->first < i) {
      const int32_t k = it->first;
      const int nk = A.rsz[k];
      std::vector<double> m = std::move(it->second);
      w.erase(it);
      apply_Ainv_right(X.Dg.blk(X.Dg.bptr[k]), X.piv.data() + X.Dg.roff[k], nk, m.data(), ni);
      if (!dropped(m.data(), ni, nk, t)) {
        for (int64_t b = X.U.bptr[k]; b < X.U.bptr[k + 1]; ++b) {
          const int32_t j = X.U.bcol[b];
          std::vector<double>& blk = w[j];
          if (blk.empty()) blk.assign((size_t)ni * A.rsz[j], 0.0);
          sub_prod(blk.data(), m.data(), X.U.blk(b), ni, nk, A.rsz[j]);
        }
        lcols.push_back(k);
        lf2.push_back(fro2(m.data(), (int64_t)ni * nk));
        lblocks.push_back(std::move(m));
      }
      it = w.upper_bound(k);
    }
    for (int k : select_lfil(lcols, lf2, lfil)) X.L.push(lcols[k], lblocks[k].data());
    X.L.end_row();
    auto d = w.find((int32_t)i);
    if (d == w.end()) return ESINGULAR;
    std::vector<int32_t> ucols;
    std::vector<double> uf2;
    std::vector<const std::vector<double>*> ublocks;
    for (auto& kv : w) {
      if (kv.first <= i) continue;
      if (dropped(kv.second.data(), ni, A.rsz[kv.first], t)) continue;
      ucols.push_back(kv.first);
      uf2.push_back(fro2(kv.second.data(), (int64_t)ni * A.rsz[kv.first]));
      ublocks.push_back(&kv.second);
    }
    for (int k : select_lfil(ucols, uf2, lfil)) X.U.push(ucols[k], ublocks[k]->data());
    X.U.end_row();
    std::vector<double> dg = d->second;
    if (gepp(dg.data(), ni, X.piv.data() + A.roff[i]) != OK) return ESINGULAR;
    X.Dg.push((int32_t)i, dg.data());
    X.Dg.end_row();
  }
  return OK;
}

// drop_all: the threshold is applied to the Schur complement at every
// reduction (the ARMS habit) instead of only at the last one (Section 3).
// fixed (optional, one flag per block row of A0): rows kept out of every
// independent set (D5); they follow the C rows from level to level.
// gs: supernodes per independent group (A1; 1 = one supernode per group);
// grouped selects the grouped factorization (A2) even for gs = 1.
int factor(const VB& A0, int nlev, double t, int lfil, double ddtol, bool drop_all, Prec& P,
           const std::vector<char>* fixed = nullptr, int gs = 1, bool grouped = false) {
  if (gs < 1) return EINVAL;
  grouped = grouped || gs > 1;
  if (A0.nbr != A0.nbc || nlev < 0 || !(t >= 0.0)) return EINVAL;
  P.n = A0.roff[A0.nbr];
  VB cur = A0;
  std::vector<char> fx;
  if (fixed) fx = *fixed;
  for (int l = 0; l < nlev && cur.nbr > 0; ++l) {
    Level L;
    L.A = cur;
    scale(L.A, L.r, L.c);
    if (grouped)
      is_order_groups(L.A, ddtol, gs, L.pI, L.nD, L.w, L.gptr, fixed ? &fx : nullptr);
    else
      is_order(L.A, ddtol, L.pI, L.nD, L.w, fixed ? &fx : nullptr);
    if (L.nD == 0) break;  // nothing to eliminate: cur becomes the last level
    const bool last_red = (l == nlev - 1) || drop_all;
    int st = grouped ? factor_level_groups(L, last_red, t, lfil) : factor_level(L, last_red, t, lfil);
    if (st != OK) return st;
    if (fixed) {
      std::vector<char> nx(L.nC);
      for (int64_t k = 0; k < L.nC; ++k) nx[k] = fx[L.pI[L.nD + k]];
      fx.swap(nx);
    }
    cur = L.S;
    P.lev.push_back(std::move(L));
  }
  if (fixed) P.last_fixed = fx;
  P.last.A = std::move(cur);
  scale(P.last.A, P.last.r, P.last.c);
  int st = ilut_last(P.last, t, lfil);
  if (st != OK) return st;
  double fill = 0;
  for (auto& L : P.lev) fill += (double)(L.D.val.size() + L.W.val.size() + L.G.val.size());
  fill += (double)(P.last.Dg.val.size() + P.last.L.val.size() + P.last.U.val.size());
  P.fill = fill;
  return OK;
}

// ---------------------------------------------------------------------------
// Solve phase, Alg. 2 (VBARMS_Solve), recursively over the levels.
// fixv (optional, D7): the values of the rows flagged in fixed, in this
// level's scaled variables before the column scaling; those rows are not
// solved for in the backward sweep.
void solve_last(const Last& X, const double* g, double* z, const double* fixv = nullptr,
                const std::vector<char>* fixed = nullptr) {
  const VB& A = X.A;
  const int64_t p = A.nbr, n = A.roff[p];
  std::vector<double> y(n);
  for (int64_t i = 0; i < n; ++i) y[i] = X.r[i] * g[i];
  // forward: y_i <- y_i - sum_{k<i} L_ik y_k
  for (int64_t i = 0; i < p; ++i) {
    const int ni = A.rsz[i];
    for (int64_t b = X.L.bptr[i]; b < X.L.bptr[i + 1]; ++b) {
      const int32_t k = X.L.bcol[b];
      const int nk = A.rsz[k];
      const double* m = X.L.blk(b);
      for (int a = 0; a < ni; ++a) {
        double s = y[A.roff[i] + a];
        for (int q = 0; q < nk; ++q) s = s - m[a * nk + q] * y[A.roff[k] + q];
        y[A.roff[i] + a] = s;
      }
    }
  }
  // backward: x_i <- D_i^{-1} (y_i - sum_{j>i} U_ij x_j)
  std::vector<double> x(n);
  for (int64_t i = p - 1; i >= 0; --i) {
    const int ni = A.rsz[i];
    if (fixv && (*fixed)[i]) {
      for (int a = 0; a < ni; ++a) x[A.roff[i] + a] = fixv[A.roff[i] + a] / X.c[A.roff[i] + a];
      continue;
    }
    std::vector<double> s(y.begin() + A.roff[i], y.begin() + A.roff[i] + ni);
    for (int64_t b = X.U.bptr[i]; b < X.U.bptr[i + 1]; ++b) {
      const int32_t j = X.U.bcol[b];
      const int nj = A.rsz[j];
      const double* u = X.U.blk(b);
      for (int a = 0; a < ni; ++a) {
        double v = s[a];
        for (int q = 0; q < nj; ++q) v = v - u[a * nj + q] * x[A.roff[j] + q];
        s[a] = v;
      }
    }
    apply_LinvP(X.Dg.blk(X.Dg.bptr[i]), X.piv.data() + A.roff[i], ni, s.data(), 1);
    apply_Uinv_left(X.Dg.blk(X.Dg.bptr[i]), ni, s.data(), 1);
    for (int a = 0; a < ni; ++a) x[A.roff[i] + a] = s[a];
  }
  for (int64_t i = 0; i < n; ++i) z[i] = X.c[i] * x[i];
}

// fixv (optional, D7): values of the fixed rows in this level's variables.
void solve_level(const Prec& P, size_t l, const double* b, double* x, const double* fixv = nullptr) {
  if (l == P.lev.size()) {
    solve_last(P.last, b, x, fixv, &P.last_fixed);
    return;
  }
  const Level& L = P.lev[l];
  const VB& A = L.A;
  const int64_t p = A.nbr, n = A.roff[p];
  // bhat = P_I S_1 b, split into f (D part) and g (C part).
  std::vector<double> bh(n);
  int64_t o = 0;
  std::vector<int64_t> newoff(p + 1, 0);
  for (int64_t k = 0; k < p; ++k) {
    const int32_t Y = L.pI[k];
    newoff[k] = o;
    for (int a = 0; a < A.rsz[Y]; ++a) bh[o + a] = L.r[A.roff[Y] + a] * b[A.roff[Y] + a];
    o += A.rsz[Y];
  }
  newoff[p] = o;
  const int64_t nf = newoff[L.nD];
  // u = L^{-1} P f (Alg. 2: solve L y = f; with groups, A3)
  std::vector<double> u(bh.begin(), bh.begin() + nf);
  for (int64_t y = 0; y < L.nD; ++y) {
    if (L.grouped) {
      const int ny = L.D.rsz[y];
      for (int64_t bb = L.Lg.bptr[y]; bb < L.Lg.bptr[y + 1]; ++bb) {
        const int32_t k = L.Lg.bcol[bb];
        const int nk = L.Lg.csz[k];
        const double* mm = L.Lg.blk(bb);
        for (int a = 0; a < ny; ++a) {
          double v = u[L.D.roff[y] + a];
          for (int q = 0; q < nk; ++q) v = v - mm[a * nk + q] * u[L.D.roff[k] + q];
          u[L.D.roff[y] + a] = v;
        }
      }
    }
    apply_LinvP(L.D.blk(L.D.bptr[y]), L.piv.data() + L.D.roff[y], L.D.rsz[y], u.data() + L.D.roff[y], 1);
  }
  // g' = g - E U^{-1} u = g - G u
  std::vector<double> g(bh.begin() + nf, bh.end());
  for (int64_t r = 0; r < L.nC; ++r) {
    const int nr = L.G.rsz[r];
    for (int64_t bb = L.G.bptr[r]; bb < L.G.bptr[r + 1]; ++bb) {
      const int32_t y = L.G.bcol[bb];
      const int m = L.G.csz[y];
      const double* gm = L.G.blk(bb);
      for (int a = 0; a < nr; ++a) {
        double s = g[L.G.roff[r] + a];
        for (int q = 0; q < m; ++q) s = s - gm[a * m + q] * u[L.G.coff[y] + q];
        g[L.G.roff[r] + a] = s;
      }
    }
  }
  // the fixed values in the next level's variables: x = c * z on the C rows
  std::vector<double> fnext;
  if (fixv) {
    fnext.assign(n - nf, 0.0);
    for (int64_t k = L.nD; k < p; ++k) {
      const int32_t Y = L.pI[k];
      for (int a = 0; a < A.rsz[Y]; ++a)
        fnext[newoff[k] - nf + a] = fixv[A.roff[Y] + a] / L.c[A.roff[Y] + a];
    }
  }
  std::vector<double> z(n - nf);
  solve_level(P, l + 1, g.data(), z.data(), fixv ? fnext.data() : nullptr);
  // y = U^{-1} (u - W z); with groups in reverse order, the group part of
  // Ubar after W (A3)
  for (int64_t yy = 0; yy < L.nD; ++yy) {
    const int64_t y = L.grouped ? L.nD - 1 - yy : yy;
    const int m = L.W.rsz[y];
    for (int64_t bb = L.W.bptr[y]; bb < L.W.bptr[y + 1]; ++bb) {
      const int32_t s = L.W.bcol[bb];
      const int ns = L.W.csz[s];
      const double* wm = L.W.blk(bb);
      for (int a = 0; a < m; ++a) {
        double v = u[L.W.roff[y] + a];
        for (int q = 0; q < ns; ++q) v = v - wm[a * ns + q] * z[L.W.coff[s] + q];
        u[L.W.roff[y] + a] = v;
      }
    }
    if (L.grouped)
      for (int64_t bb = L.Ug.bptr[y]; bb < L.Ug.bptr[y + 1]; ++bb) {
        const int32_t j = L.Ug.bcol[bb];
        const int nj = L.Ug.csz[j];
        const double* um = L.Ug.blk(bb);
        for (int a = 0; a < m; ++a) {
          double v = u[L.D.roff[y] + a];
          for (int q = 0; q < nj; ++q) v = v - um[a * nj + q] * u[L.D.roff[j] + q];
          u[L.D.roff[y] + a] = v;
        }
      }
    apply_Uinv_left(L.D.blk(L.D.bptr[y]), m, u.data() + L.D.roff[y], 1);
  }
  // x = S_2 P_I^T [y; z]
  for (int64_t k = 0; k < p; ++k) {
    const int32_t Y = L.pI[k];
    for (int a = 0; a < A.rsz[Y]; ++a) {
      const double v = k < L.nD ? u[newoff[k] + a] : z[newoff[k] - nf + a];
      x[A.roff[Y] + a] = L.c[A.roff[Y] + a] * v;
    }
  }
}

void spmv(const VB& A, const double* x, double* y) {
  for (int64_t I = 0; I < A.nbr; ++I) {
    const int m = A.rsz[I];
    for (int a = 0; a < m; ++a) {
      double s = 0.0;
      for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
        const int32_t J = A.bcol[b];
        const int nc = A.csz[J];
        const double* v = A.blk(b);
        for (int q = 0; q < nc; ++q) s = s + v[a * nc + q] * x[A.coff[J] + q];
      }
      y[A.roff[I] + a] = s;
    }
  }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s = s + a[i] * b[i];
  return s;
}

// ---------------------------------------------------------------------------
// Section 5: global preconditioners with VBARMS as the local solver (block
// Jacobi, Schwarz), all subdomains in one address space (D1-D3).
struct DD {
  int nparts = 0, delta = 0;
  bool restricted = true;
  int64_t n = 0;
  std::vector<int64_t> roff;            // scalar offsets of A's block rows
  std::vector<int32_t> part;            // W_i^0 membership of each block row
  std::vector<std::vector<int32_t>> W;  // W_i^delta, ascending block rows of A
  std::vector<VB> Aloc;                 // A_i = R_i A R_i on W_i^delta
  std::vector<Prec> loc;                // VBARMS of A_i
};

int dd_build(const VB& A, int nparts, int delta, bool restricted, int nlev, double t, int lfil, double ddtol,
             bool drop_all, DD& D) {
  if (A.nbr != A.nbc || nparts < 1 || delta < 0) return EINVAL;
  const int64_t p = A.nbr, n = A.roff[p];
  D.nparts = nparts;
  D.delta = delta;
  D.restricted = restricted;
  D.n = n;
  D.roff = A.roff;
  // D1: contiguous ranges of block rows of near-equal scalar size
  D.part.assign(p, 0);
  for (int64_t I = 0; I < p; ++I) D.part[I] = (int32_t)(((int64_t)nparts * A.roff[I]) / n);
  // D2: the block graph of A + A^T
  std::vector<std::vector<int32_t>> adj(p);
  for (int64_t I = 0; I < p; ++I)
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      adj[I].push_back(A.bcol[b]);
      adj[A.bcol[b]].push_back((int32_t)I);
    }
  D.W.assign(nparts, {});
  D.Aloc.assign(nparts, VB());
  D.loc.assign(nparts, Prec());
  for (int i = 0; i < nparts; ++i) {
    std::vector<char> in(p, 0);
    for (int64_t I = 0; I < p; ++I) in[I] = D.part[I] == i;
    for (int d = 0; d < delta; ++d) {  // W_i^d = adj(W_i^{d-1})
      std::vector<char> next = in;
      for (int64_t I = 0; I < p; ++I)
        if (in[I])
          for (int32_t J : adj[I]) next[J] = 1;
      in.swap(next);
    }
    std::vector<int32_t>& Wi = D.W[i];
    std::vector<int32_t> local(p, -1);
    for (int64_t I = 0; I < p; ++I)
      if (in[I]) {
        local[I] = (int32_t)Wi.size();
        Wi.push_back((int32_t)I);
      }
    std::vector<int32_t> sz;
    for (int32_t I : Wi) sz.push_back(A.rsz[I]);
    VB& Ai = D.Aloc[i];
    Ai.init(sz, sz);
    for (int32_t I : Wi) {
      for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b)
        if (local[A.bcol[b]] >= 0) Ai.push(local[A.bcol[b]], A.blk(b));
      Ai.end_row();
    }
    if (Wi.empty()) continue;
    const int st = factor(Ai, nlev, t, lfil, ddtol, drop_all, D.loc[i]);
    if (st != OK) return st;
  }
  return OK;
}

// D3: y = sum_i Q_i^T A_i^{-1} R_i x with A_i^{-1} the local VBARMS solve;
// Q_i = R_i (additive Schwarz; block Jacobi when delta = 0) or the restriction
// to W_i^0 (restricted additive Schwarz).  Subdomains are added in order.
void dd_apply(const DD& D, const double* x, double* y) {
  for (int64_t j = 0; j < D.n; ++j) y[j] = 0.0;
  for (int i = 0; i < D.nparts; ++i) {
    const std::vector<int32_t>& Wi = D.W[i];
    if (Wi.empty()) continue;
    const VB& Ai = D.Aloc[i];
    std::vector<double> xi(Ai.roff[Ai.nbr]), zi(Ai.roff[Ai.nbr]);
    for (size_t k = 0; k < Wi.size(); ++k)
      for (int a = 0; a < Ai.rsz[k]; ++a) xi[Ai.roff[k] + a] = x[D.roff[Wi[k]] + a];
    solve_level(D.loc[i], 0, xi.data(), zi.data());
    for (size_t k = 0; k < Wi.size(); ++k) {
      if (D.restricted && D.part[Wi[k]] != i) continue;
      for (int a = 0; a < Ai.rsz[k]; ++a) y[D.roff[Wi[k]] + a] = y[D.roff[Wi[k]] + a] + zi[Ai.roff[k] + a];
    }
  }
}

// Section 5, Schur-complement global preconditioner (D4-D7), all subdomains
// in one address space.
struct DDS {
  int nparts = 0, msteps = 0;
  int64_t n = 0, ng = 0;
  std::vector<int64_t> roff;            // scalar offsets of A's block rows
  std::vector<int32_t> part;            // D1
  std::vector<char> iface;              // D4, per block row of A
  std::vector<std::vector<int32_t>> W;  // subdomain rows: interior, then interface
  std::vector<int64_t> nint;            // interior block rows per subdomain
  std::vector<int64_t> gofs;            // start of each subdomain's interface in the global interface vector
  std::vector<VB> Aloc;                 // A_i (D4)
  std::vector<Prec> loc;                // VBARMS of A_i with fixed interface (D5)
  VB E;                                 // E_ij on the global interface numbering
};

int dds_build(const VB& A, int nparts, int msteps, int nlev, double t, int lfil, double ddtol, bool drop_all,
              DDS& D) {
  if (A.nbr != A.nbc || nparts < 1 || msteps < 1) return EINVAL;
  const int64_t p = A.nbr, n = A.roff[p];
  D.nparts = nparts;
  D.msteps = msteps;
  D.n = n;
  D.roff = A.roff;
  D.part.assign(p, 0);
  for (int64_t I = 0; I < p; ++I) D.part[I] = (int32_t)(((int64_t)nparts * A.roff[I]) / n);
  // D4: interface rows
  D.iface.assign(p, 0);
  for (int64_t I = 0; I < p; ++I)
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      const int32_t J = A.bcol[b];
      if (D.part[J] != D.part[I]) {
        D.iface[I] = 1;
        D.iface[J] = 1;
      }
    }
  D.W.assign(nparts, {});
  D.nint.assign(nparts, 0);
  D.Aloc.assign(nparts, VB());
  D.loc.assign(nparts, Prec());
  std::vector<int32_t> local(p, -1);
  for (int i = 0; i < nparts; ++i) {
    std::vector<int32_t>& Wi = D.W[i];
    for (int64_t I = 0; I < p; ++I)
      if (D.part[I] == i && !D.iface[I]) Wi.push_back((int32_t)I);
    D.nint[i] = (int64_t)Wi.size();
    for (int64_t I = 0; I < p; ++I)
      if (D.part[I] == i && D.iface[I]) Wi.push_back((int32_t)I);
    for (size_t k = 0; k < Wi.size(); ++k) local[Wi[k]] = (int32_t)k;
  }
  for (int i = 0; i < nparts; ++i) {
    const std::vector<int32_t>& Wi = D.W[i];
    if (Wi.empty()) continue;
    std::vector<int32_t> sz;
    for (int32_t I : Wi) sz.push_back(A.rsz[I]);
    VB& Ai = D.Aloc[i];
    Ai.init(sz, sz);
    for (int32_t I : Wi) {
      std::vector<std::pair<int32_t, int64_t>> blks;  // (local column, block of A)
      for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b)
        if (D.part[A.bcol[b]] == i) blks.push_back({local[A.bcol[b]], b});
      std::sort(blks.begin(), blks.end());
      for (auto& cb : blks) Ai.push(cb.first, A.blk(cb.second));
      Ai.end_row();
    }
    std::vector<char> fixed(Wi.size(), 0);
    for (size_t k = (size_t)D.nint[i]; k < Wi.size(); ++k) fixed[k] = 1;
    const int st = factor(Ai, nlev, t, lfil, ddtol, drop_all, D.loc[i], &fixed);
    if (st != OK) return st;
  }
  // the global interface vector: every subdomain's interface rows in turn
  std::vector<int32_t> gpos(p, -1), gsz;
  D.gofs.assign(nparts + 1, 0);
  int64_t o = 0;
  for (int i = 0; i < nparts; ++i) {
    D.gofs[i] = o;
    for (size_t k = (size_t)D.nint[i]; k < D.W[i].size(); ++k) {
      gpos[D.W[i][k]] = (int32_t)gsz.size();
      gsz.push_back(A.rsz[D.W[i][k]]);
      o += A.rsz[D.W[i][k]];
    }
  }
  D.gofs[nparts] = o;
  D.ng = o;
  // E: the blocks of A between interface rows of different subdomains
  D.E.init(gsz, gsz);
  for (int i = 0; i < nparts; ++i)
    for (size_t k = (size_t)D.nint[i]; k < D.W[i].size(); ++k) {
      const int32_t I = D.W[i][k];
      std::vector<std::pair<int32_t, int64_t>> blks;
      for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b)
        if (D.part[A.bcol[b]] != i) blks.push_back({gpos[A.bcol[b]], b});
      std::sort(blks.begin(), blks.end());
      for (auto& cb : blks) D.E.push(cb.first, A.blk(cb.second));
      D.E.end_row();
    }
  return OK;
}

// Local solve of subdomain i: r in A's numbering (or, when rloc, already in
// the subdomain's), result in the subdomain's numbering.
void dds_local_solve(const DDS& D, int i, const double* r, bool rloc, std::vector<double>& out,
                     const double* fixv = nullptr) {
  const VB& Ai = D.Aloc[i];
  const int64_t ni = Ai.roff[Ai.nbr];
  std::vector<double> ri(ni);
  if (rloc) {
    for (int64_t q = 0; q < ni; ++q) ri[q] = r[q];
  } else {
    for (size_t k = 0; k < D.W[i].size(); ++k)
      for (int a = 0; a < Ai.rsz[k]; ++a) ri[Ai.roff[k] + a] = r[D.roff[D.W[i][k]] + a];
  }
  out.assign(ni, 0.0);
  solve_level(D.loc[i], 0, ri.data(), out.data(), fixv);
}

// out = blockdiag(S_i)^{-1} v on the global interface vector (D6).
void dds_sinv(const DDS& D, const double* v, double* out) {
  for (int i = 0; i < D.nparts; ++i) {
    const VB& Ai = D.Aloc[i];
    if (D.W[i].empty()) continue;
    const int64_t ni = Ai.roff[Ai.nbr], i0 = Ai.roff[D.nint[i]];
    std::vector<double> ri(ni, 0.0), zi;
    for (int64_t q = i0; q < ni; ++q) ri[q] = v[D.gofs[i] + q - i0];
    dds_local_solve(D, i, ri.data(), true, zi);
    for (int64_t q = i0; q < ni; ++q) out[D.gofs[i] + q - i0] = zi[q];
  }
}

// D6: msteps steps of GMRES with y_0 = 0 on op(y) = z.
void gmres_steps(const std::function<void(const double*, double*)>& op, const std::vector<double>& z, int m,
                 std::vector<double>& y) {
  const size_t n = z.size();
  y.assign(n, 0.0);
  const double beta = std::sqrt(dot(z, z));
  if (beta == 0.0) return;
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n));
  std::vector<double> w(n), H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1, 0.0), yv(m);
  for (size_t q = 0; q < n; ++q) V[0][q] = z[q] / beta;
  gv[0] = beta;
  int j = 0;
  for (; j < m; ++j) {
    op(V[j].data(), w.data());
    for (int i = 0; i <= j; ++i) {
      const double h = dot(w, V[i]);
      H[(size_t)i * m + j] = h;
      for (size_t q = 0; q < n; ++q) w[q] = w[q] - h * V[i][q];
    }
    const double hn = std::sqrt(dot(w, w));
    H[(size_t)(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
      H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
      H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
    }
    const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
    const double d = std::sqrt(a * a + c * c);
    cs[j] = d > 0.0 ? a / d : 1.0;
    sn[j] = d > 0.0 ? c / d : 0.0;
    H[(size_t)j * m + j] = d;
    H[(size_t)(j + 1) * m + j] = 0.0;
    gv[j + 1] = -sn[j] * gv[j];
    gv[j] = cs[j] * gv[j];
    if (hn == 0.0) {
      ++j;
      break;
    }
    for (size_t q = 0; q < n; ++q) V[j + 1][q] = w[q] / hn;
  }
  for (int i = j - 1; i >= 0; --i) {
    double sacc = gv[i];
    for (int k = i + 1; k < j; ++k) sacc = sacc - H[(size_t)i * m + k] * yv[k];
    yv[i] = H[(size_t)i * m + i] != 0.0 ? sacc / H[(size_t)i * m + i] : 0.0;
  }
  for (int i = 0; i < j; ++i)
    for (size_t q = 0; q < n; ++q) y[q] = y[q] + yv[i] * V[i][q];
}

// One application y = M^{-1} x (D6, D7), both in A's numbering.
void dds_apply(const DDS& D, const double* x, double* yout) {
  std::vector<double> z(D.ng), yg;
  std::vector<double> zi;
  for (int i = 0; i < D.nparts; ++i) {  // z_i = S_i^{-1} g'_i
    if (D.W[i].empty()) continue;
    dds_local_solve(D, i, x, false, zi);
    const VB& Ai = D.Aloc[i];
    const int64_t ni = Ai.roff[Ai.nbr], i0 = Ai.roff[D.nint[i]];
    for (int64_t q = i0; q < ni; ++q) z[D.gofs[i] + q - i0] = zi[q];
  }
  auto op = [&D](const double* v, double* out) {  // v + S^{-1} E v
    std::vector<double> w(D.ng), t(D.ng);
    spmv(D.E, v, w.data());
    dds_sinv(D, w.data(), t.data());
    for (int64_t q = 0; q < D.ng; ++q) out[q] = v[q] + t[q];
  };
  gmres_steps(op, z, D.msteps, yg);
  for (int i = 0; i < D.nparts; ++i) {  // u_i = B_i^{-1} (f_i - F_i y_i)
    if (D.W[i].empty()) continue;
    const VB& Ai = D.Aloc[i];
    const int64_t ni = Ai.roff[Ai.nbr], i0 = Ai.roff[D.nint[i]];
    std::vector<double> fv(ni, 0.0), ui;
    for (int64_t q = i0; q < ni; ++q) fv[q] = yg[D.gofs[i] + q - i0];
    dds_local_solve(D, i, x, false, ui, fv.data());
    for (size_t k = 0; k < D.W[i].size(); ++k)
      for (int a = 0; a < Ai.rsz[k]; ++a)
        yout[D.roff[D.W[i][k]] + a] = (int64_t)k < D.nint[i] ? ui[Ai.roff[k] + a] : fv[Ai.roff[k] + a];
  }
}

// R9: flexible GMRES(m) with right preconditioning (FGMRES, Saad 1993).
using PrecFn = std::function<void(const double*, double*)>;  // z = M^{-1} v; empty: M = I
int fgmres(const VB& A, const PrecFn& P, const double* b, double* x, double rtol, int m, int maxit, int* iters,
           double* relres) {
  const int64_t n = A.roff[A.nbr];
  std::vector<double> bv(b, b + n), r(n), w(n);
  const double bnorm = std::sqrt(dot(bv, bv));
  *iters = 0;
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    return OK;
  }
  const double target = rtol * bnorm;
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), yv(m);
  int it = 0;
  double rnorm = 0.0;
  for (;;) {
    spmv(A, x, w.data());
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    rnorm = std::sqrt(dot(r, r));
    if (rnorm <= target || it >= maxit) break;
    for (int64_t i = 0; i < n; ++i) V[0][i] = r[i] / rnorm;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = rnorm;
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      if (P)
        P(V[j].data(), Z[j].data());
      else
        Z[j] = V[j];
      spmv(A, Z[j].data(), w.data());
      for (int i = 0; i <= j; ++i) {
        double h = dot(w, V[i]);
        H[(size_t)i * m + j] = h;
        for (int64_t q = 0; q < n; ++q) w[q] = w[q] - h * V[i][q];
      }
      const double hn = std::sqrt(dot(w, w));
      H[(size_t)(j + 1) * m + j] = hn;
      ++it;
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double d = std::sqrt(a * a + c * c);
      cs[j] = d > 0.0 ? a / d : 1.0;
      sn[j] = d > 0.0 ? c / d : 0.0;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      if (hn == 0.0 || std::fabs(gv[j + 1]) <= target) {
        ++j;
        break;
      }
      for (int64_t q = 0; q < n; ++q) V[j + 1][q] = w[q] / hn;
    }
    // x <- x + Z y with H(0:j,0:j) y = g(0:j)
    for (int i = j - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k = i + 1; k < j; ++k) s = s - H[(size_t)i * m + k] * yv[k];
      yv[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
    }
    for (int i = 0; i < j; ++i)
      for (int64_t q = 0; q < n; ++q) x[q] = x[q] + yv[i] * Z[i][q];
  }
  *iters = it;
  *relres = rnorm / bnorm;
  return rnorm <= target ? OK : ENOCONV;
}

thread_local int g_last_status = 0;

}  // namespace

// ===========================================================================
// C interface for the test suite (ctypes).  Handles are heap objects.
extern "C" {

struct or_cmp;
struct or_prec;

int or_last_status() { return g_last_status; }

void* or_compress(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau) {
  auto* c = new Compressed();
  g_last_status = compress(n, rowptr, colind, val, tau, *c);
  if (g_last_status != OK) {
    delete c;
    return nullptr;
  }
  return c;
}
void* or_compress_two_pass(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau) {
  auto* c = new Compressed();
  g_last_status = compress_two_pass(n, rowptr, colind, val, tau, *c);
  if (g_last_status != OK) {
    delete c;
    return nullptr;
  }
  return c;
}
void* or_graph_compress(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double mu) {
  auto* c = new Compressed();
  g_last_status = graph_compress(n, rowptr, colind, val, mu, *c);
  if (g_last_status != OK) {
    delete c;
    return nullptr;
  }
  return c;
}
void or_cmp_free(void* h) { delete (Compressed*)h; }
int64_t or_cmp_nblk(void* h) { return (int64_t)((Compressed*)h)->bsz.size(); }
void or_cmp_perm(void* h, int32_t* perm, int32_t* bsz) {
  auto* c = (Compressed*)h;
  std::copy(c->perm.begin(), c->perm.end(), perm);
  std::copy(c->bsz.begin(), c->bsz.end(), bsz);
}
void or_cmp_quality(void* h, double* av_bd, double* av_bs) {
  *av_bd = ((Compressed*)h)->av_bd;
  *av_bs = ((Compressed*)h)->av_bs;
}
const void* or_cmp_matrix(void* h) { return &((Compressed*)h)->A; }

// VBCSR matrices: create from arrays, query, export.
void* or_vb_create(int64_t nbr, int64_t nbc, const int32_t* rsz, const int32_t* csz, const int64_t* bptr,
                   const int32_t* bcol, const int64_t* voff, const double* val) {
  auto* m = new VB();
  m->init(std::vector<int32_t>(rsz, rsz + nbr), std::vector<int32_t>(csz, csz + nbc));
  for (int64_t I = 0; I < nbr; ++I) {
    for (int64_t b = bptr[I]; b < bptr[I + 1]; ++b) m->push(bcol[b], val + voff[b]);
    m->end_row();
  }
  return m;
}
void or_vb_free(void* h) { delete (VB*)h; }
void or_vb_dims(const void* h, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval) {
  const VB* m = (const VB*)h;
  *nbr = m->nbr;
  *nbc = m->nbc;
  *nnzb = m->nnzb();
  *nval = (int64_t)m->val.size();
}
void or_vb_export(const void* h, int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff,
                  double* val) {
  const VB* m = (const VB*)h;
  std::copy(m->rsz.begin(), m->rsz.end(), rsz);
  std::copy(m->csz.begin(), m->csz.end(), csz);
  std::copy(m->bptr.begin(), m->bptr.end(), bptr);
  std::copy(m->bcol.begin(), m->bcol.end(), bcol);
  std::copy(m->voff.begin(), m->voff.end(), voff);
  std::copy(m->val.begin(), m->val.end(), val);
}
void or_vb_spmv(const void* h, const double* x, double* y) { spmv(*(const VB*)h, x, y); }

// Step 2 and Step 3 on their own (for checks on identical input).
void or_scale(void* h, double* r, double* c) {
  VB* m = (VB*)h;
  std::vector<double> rv, cv;
  scale(*m, rv, cv);
  std::copy(rv.begin(), rv.end(), r);
  std::copy(cv.begin(), cv.end(), c);
}
int64_t or_is_order(const void* h, double ddtol, int32_t* pI, double* w) {
  std::vector<int32_t> p;
  std::vector<double> wv;
  int64_t nD = 0;
  is_order(*(const VB*)h, ddtol, p, nD, wv);
  std::copy(p.begin(), p.end(), pI);
  std::copy(wv.begin(), wv.end(), w);
  return nD;
}
int or_gepp(double* a, int m, int32_t* piv) { return gepp(a, m, piv); }
int or_dropped(const double* a, int m, int n, double t) { return dropped(a, m, n, t) ? 1 : 0; }

void* or_factor(const void* A, int nlev, double droptol, int lfil, double ddtol, int drop_all) {
  auto* P = new Prec();
  g_last_status = factor(*(const VB*)A, nlev, droptol, lfil, ddtol, drop_all != 0, *P);
  if (g_last_status != OK) {
    delete P;
    return nullptr;
  }
  return P;
}
// With groups of up to gs supernodes (A1, A2); grouped != 0 takes the grouped
// code even for gs = 1.
void* or_factor_groups(const void* A, int nlev, double droptol, int lfil, double ddtol, int drop_all, int gs,
                       int grouped) {
  auto* P = new Prec();
  g_last_status = factor(*(const VB*)A, nlev, droptol, lfil, ddtol, drop_all != 0, *P, nullptr, gs, grouped != 0);
  if (g_last_status != OK) {
    delete P;
    return nullptr;
  }
  return P;
}
int64_t or_prec_gptr(void* h, int l, int64_t* out) {
  const Level& L = ((Prec*)h)->lev[l];
  if (out) std::copy(L.gptr.begin(), L.gptr.end(), out);
  return (int64_t)L.gptr.size();
}
// The same with fixed rows (D5): fixed[nbr] flags, or NULL.
void* or_factor_fixed(const void* A, int nlev, double droptol, int lfil, double ddtol, int drop_all,
                      const int32_t* fixed) {
  const VB& M = *(const VB*)A;
  std::vector<char> fx;
  if (fixed)
    for (int64_t I = 0; I < M.nbr; ++I) fx.push_back(fixed[I] != 0);
  auto* P = new Prec();
  g_last_status = factor(M, nlev, droptol, lfil, ddtol, drop_all != 0, *P, fixed ? &fx : nullptr);
  if (g_last_status != OK) {
    delete P;
    return nullptr;
  }
  return P;
}
void or_prec_free(void* h) { delete (Prec*)h; }
int or_prec_levels(void* h) { return (int)((Prec*)h)->lev.size(); }
double or_prec_fill(void* h) { return ((Prec*)h)->fill; }
int64_t or_prec_nd(void* h, int l) { return ((Prec*)h)->lev[l].nD; }
// which: 0 scaled A, 1 D (pivot LU), 2 F, 3 E, 4 C, 5 W, 6 G, 7 S, 10 group
// multipliers, 11 group part of Ubar (grouped levels);
// for l == levels (last level): 0 scaled A, 1 pivot LU, 8 L, 9 U.
const void* or_prec_mat(void* h, int l, int which) {
  Prec* P = (Prec*)h;
  if (l == (int)P->lev.size()) {
    switch (which) {
      case 0: return &P->last.A;
      case 1: return &P->last.Dg;
      case 8: return &P->last.L;
      case 9: return &P->last.U;
    }
    return nullptr;
  }
  Level& L = P->lev[l];
  switch (which) {
    case 0: return &L.A;
    case 1: return &L.D;
    case 2: return &L.F;
    case 3: return &L.E;
    case 4: return &L.C;
    case 5: return &L.W;
    case 6: return &L.G;
    case 7: return &L.S;
    case 10: return L.grouped ? &L.Lg : nullptr;
    case 11: return L.grouped ? &L.Ug : nullptr;
  }
  return nullptr;
}
// Vectors: 0 r, 1 c, 2 w (doubles); 3 pI, 4 piv (int32).  Returns length.
int64_t or_prec_vec(void* h, int l, int which, double* dout, int32_t* iout) {
  Prec* P = (Prec*)h;
  const bool last = l == (int)P->lev.size();
  const std::vector<double>* dv = nullptr;
  const std::vector<int32_t>* iv = nullptr;
  if (last) {
    if (which == 0) dv = &P->last.r;
    if (which == 1) dv = &P->last.c;
    if (which == 4) iv = &P->last.piv;
  } else {
    Level& L = P->lev[l];
    if (which == 0) dv = &L.r;
    if (which == 1) dv = &L.c;
    if (which == 2) dv = &L.w;
    if (which == 3) iv = &L.pI;
    if (which == 4) iv = &L.piv;
  }
  if (dv) {
    if (dout) std::copy(dv->begin(), dv->end(), dout);
    return (int64_t)dv->size();
  }
  if (iv) {
    if (iout) std::copy(iv->begin(), iv->end(), iout);
    return (int64_t)iv->size();
  }
  return -1;
}
void or_apply(void* h, const double* b, double* x) { solve_level(*(Prec*)h, 0, b, x); }
int or_fgmres(const void* A, void* prec, const double* b, double* x, double rtol, int m, int maxit, int* iters,
              double* relres) {
  PrecFn M;
  if (prec) M = [prec](const double* v, double* z) { solve_level(*(const Prec*)prec, 0, v, z); };
  return fgmres(*(const VB*)A, M, b, x, rtol, m, maxit, iters, relres);
}

void* or_dd_build(const void* A, int nparts, int delta, int restricted, int nlev, double t, int lfil, double ddtol,
                  int drop_all) {
  auto* D = new DD();
  g_last_status = dd_build(*(const VB*)A, nparts, delta, restricted != 0, nlev, t, lfil, ddtol, drop_all != 0, *D);
  if (g_last_status != OK) {
    delete D;
    return nullptr;
  }
  return D;
}
void or_dd_free(void* h) { delete (DD*)h; }
int64_t or_dd_part(void* h, int32_t* part) {
  const DD* D = (const DD*)h;
  if (part) std::copy(D->part.begin(), D->part.end(), part);
  return (int64_t)D->part.size();
}
int64_t or_dd_rows(void* h, int i, int32_t* rows) {
  const DD* D = (const DD*)h;
  if (rows) std::copy(D->W[i].begin(), D->W[i].end(), rows);
  return (int64_t)D->W[i].size();
}
const void* or_dd_local(void* h, int i) { return &((DD*)h)->Aloc[i]; }
void* or_dd_local_prec(void* h, int i) { return &((DD*)h)->loc[i]; }
void or_dd_apply(void* h, const double* x, double* y) { dd_apply(*(const DD*)h, x, y); }
int or_dd_fgmres(const void* A, void* h, const double* b, double* x, double rtol, int m, int maxit, int* iters,
                 double* relres) {
  const DD* D = (const DD*)h;
  PrecFn M = [D](const double* v, double* z) { dd_apply(*D, v, z); };
  return fgmres(*(const VB*)A, M, b, x, rtol, m, maxit, iters, relres);
}


void* or_dds_build(const void* A, int nparts, int msteps, int nlev, double t, int lfil, double ddtol, int drop_all) {
  auto* D = new DDS();
  g_last_status = dds_build(*(const VB*)A, nparts, msteps, nlev, t, lfil, ddtol, drop_all != 0, *D);
  if (g_last_status != OK) {
    delete D;
    return nullptr;
  }
  return D;
}
void or_dds_free(void* h) { delete (DDS*)h; }
int64_t or_dds_iface(void* h, int32_t* part, int32_t* iface) {
  const DDS* D = (const DDS*)h;
  for (size_t I = 0; I < D->part.size(); ++I) {
    if (part) part[I] = D->part[I];
    if (iface) iface[I] = D->iface[I];
  }
  return (int64_t)D->part.size();
}
int64_t or_dds_rows(void* h, int i, int32_t* rows, int64_t* nint) {
  const DDS* D = (const DDS*)h;
  if (rows) std::copy(D->W[i].begin(), D->W[i].end(), rows);
  if (nint) *nint = D->nint[i];
  return (int64_t)D->W[i].size();
}
const void* or_dds_local(void* h, int i) { return &((DDS*)h)->Aloc[i]; }
void* or_dds_local_prec(void* h, int i) { return &((DDS*)h)->loc[i]; }
const void* or_dds_coupling(void* h) { return &((DDS*)h)->E; }
int64_t or_dds_ng(void* h) { return ((DDS*)h)->ng; }
void or_dds_sinv(void* h, const double* v, double* out) { dds_sinv(*(const DDS*)h, v, out); }
void or_dds_apply(void* h, const double* x, double* y) { dds_apply(*(const DDS*)h, x, y); }
int or_dds_fgmres(const void* A, void* h, const double* b, double* x, double rtol, int m, int maxit, int* iters,
                  double* relres) {
  const DDS* D = (const DDS*)h;
  PrecFn M = [D](const double* v, double* z) { dds_apply(*D, v, z); };
  return fgmres(*(const VB*)A, M, b, x, rtol, m, maxit, iters, relres);
}
int64_t or_prec_last_fixed(void* h, int32_t* out) {
  const Prec* P = (const Prec*)h;
  if (out)
    for (size_t k = 0; k < P->last_fixed.size(); ++k) out[k] = P->last_fixed[k];
  return (int64_t)P->last_fixed.size();
}

}  // extern "C"
