/*
 * xref.c -- CPU FP64 oracle for the crossbar nodal solve of XbarSim
 * (Kolinko, Amin, Zand, Bakos, arXiv 2410.19993).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, step by step in the paper's order:
 *   1. xref_assemble_band: the 2MN x 2MN nodal conductance matrix of an
 *      M x N crossbar (Sec. II-A "Circuit Model", KCL Eqs. 1-4 and the nodal
 *      equations Eqs. 5-7), written in the interleaved unknown ordering of
 *      Sec. II-B "Matrix Formulation" (WL(1,1), BL(1,1), WL(1,2), BL(1,2), ...),
 *      which makes the matrix banded with half-bandwidth 2N.  Stored as a band.
 *   2. xref_rhs: the nodal current vector, nonzero only at the word-line nodes
 *      driven by the input sources (Eq. 5 right-hand side).
 *   3. xref_lu_band: LU decomposition G = LU with L unit lower triangular
 *      (Sec. II-C "Solution Cost").  Plain Gaussian elimination restricted to
 *      the band, no pivoting (see below).
 *   4. xref_solve_band: forward substitution L y = I, then back substitution
 *      U V = y, for every right-hand side of a batch (Sec. II-C; one
 *      decomposition serves a whole batch, Sec. III-A).
 *   5. xref_extract: bit-line termination currents (Sec. II "Methodology":
 *      the current through the termination of each BL is the output), the
 *      node voltages, and the source currents.
 *
 * Readings of the paper (each is listed in the design notes):
 *   - Source V_i drives WL(i,1) through R_s (Eq. 5 uses G_WL for this
 *     segment; here g_s = 1/R_s, and R_s = R_w reproduces the paper).  The far
 *     end WL(i,N) is open (Eq. 2).  The top of each bit line, BL(1,j), is open
 *     (Eq. 3).  The bottom BL(M,j) is tied to ground through R_sense; its
 *     current g_o*V_BL(M,j) is the output I_j (g_o = 1/R_sense).
 *   - Word-line segments R_w sit between adjacent columns, bit-line segments
 *     R_b between adjacent rows.
 *   - Eq. 7's coefficient "s(-G_D(i,j))" and range "1<j<m" are typos; the BL
 *     row couples to WL(i,j) with -G_ij for every j.
 *
 * No pivoting: the nodal matrix is symmetric, irreducibly diagonally dominant
 * with nonpositive off-diagonals (a nonsingular M-matrix), so Gaussian
 * elimination with partial pivoting would pick the diagonal at every step
 * (column diagonal dominance is preserved by elimination; Golub & Van Loan,
 * Matrix Computations, Sec. 3.4).  Elimination without interchanges therefore
 * performs exactly the decomposition the paper's LU computes.
 *
 * Build with -ffp-contract=off so results do not depend on FMA contraction.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* index of WL(i,j) and BL(i,j), 0-based i<M, j<N, interleaved (Sec. II-B) */
static size_t idx_wl(int N, int i, int j) { return 2 * ((size_t)i * (size_t)N + (size_t)j); }
static size_t idx_bl(int N, int i, int j) { return idx_wl(N, i, j) + 1; }

int xref_half_bandwidth(int M, int N) { (void)M; return 2 * N; }

/* band storage: row r holds entries c in [r-p, r+p] at a[r*(2p+1) + (c-r+p)] of a k x k matrix.
 * An entry outside the matrix or outside the band is not stored and marks the assembly as
 * failed: a wrong node index must fail loudly instead of writing past the array. */
typedef struct {
  double* a;
  size_t k;
  int bad;
} Band;

static void band_add(Band* ab, int p, size_t r, size_t c, double v) {
  const long long d = (long long)c - (long long)r;
  if (r >= ab->k || c >= ab->k || d < -p || d > p) {
    ab->bad = 1;
    return;
  }
  ab->a[r * (size_t)(2 * p + 1) + (size_t)(d + p)] += v;
}

/*
 * Assemble the nodal matrix (Eqs. 1-7) into band storage ab[(2MN) x (4N+1)].
 * G is M x N row-major (G[i*N+j] is the conductance of device D(i,j)).
 * Each row is the KCL equation of its node written as
 *   (sum of conductances at the node) * V_node - sum_k g_k * V_neighbour_k = injected current.
 * Returns 0, -1 on invalid arguments, or -2 if a node index fell outside the matrix or band.
 */
int xref_assemble_band(int M, int N, const double* G, double Rs, double Rw, double Rb,
                       double Rsense, double* abuf) {
  if (M < 1 || N < 1 || !G || !abuf) return -1;
  if (!(Rs > 0) || !(Rw > 0) || !(Rb > 0) || !(Rsense > 0)) return -1;
  const double gs = 1.0 / Rs, gw = 1.0 / Rw, gb = 1.0 / Rb, go = 1.0 / Rsense;
  const int p = 2 * N;
  const size_t k = 2 * (size_t)M * (size_t)N;
  memset(abuf, 0, k * (size_t)(2 * p + 1) * sizeof(double));
  Band band = {abuf, k, 0};
  Band* ab = &band;
  for (int i = 0; i < M; ++i) {
    for (int j = 0; j < N; ++j) {
      const double g = G[(size_t)i * N + j];
      const size_t w = idx_wl(N, i, j), u = idx_bl(N, i, j);
      /* word-line node WL(i,j): Eq. 5 (j = 1), Eq. 6 (interior), Eq. 2 (j = N, open end) */
      band_add(ab, p, w, w, g);          /* memristor D(i,j) to BL(i,j) */
      band_add(ab, p, w, u, -g);
      if (j == 0) {
        band_add(ab, p, w, w, gs);       /* source segment to V_i (right-hand side) */
      } else {
        band_add(ab, p, w, w, gw);       /* segment to WL(i,j-1) */
        band_add(ab, p, w, idx_wl(N, i, j - 1), -gw);
      }
      if (j < N - 1) {
        band_add(ab, p, w, w, gw);       /* segment to WL(i,j+1) */
        band_add(ab, p, w, idx_wl(N, i, j + 1), -gw);
      }
      /* bit-line node BL(i,j): Eq. 3 (i = 1, open top), Eq. 7 (interior), termination at i = M */
      band_add(ab, p, u, u, g);
      band_add(ab, p, u, w, -g);
      if (i > 0) {
        band_add(ab, p, u, u, gb);       /* segment to BL(i-1,j) */
        band_add(ab, p, u, idx_bl(N, i - 1, j), -gb);
      }
      if (i < M - 1) {
        band_add(ab, p, u, u, gb);       /* segment to BL(i+1,j) */
        band_add(ab, p, u, idx_bl(N, i + 1, j), -gb);
      } else {
        band_add(ab, p, u, u, go);       /* sense resistor to ground */
      }
    }
  }
  return band.bad ? -2 : 0;
}

/*
 * Right-hand sides for a batch of B input vectors V[B x M] (row b is one input
 * vector): rhs[b*2MN + node] = g_s * V_i at WL(i,1), zero elsewhere (Eq. 5).
 */
int xref_rhs(int M, int N, int B, const double* V, double Rs, double* rhs) {
  if (M < 1 || N < 1 || B < 0 || !(Rs > 0)) return -1;
  const size_t k = 2 * (size_t)M * (size_t)N;
  memset(rhs, 0, (size_t)B * k * sizeof(double));
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < M; ++i) rhs[(size_t)b * k + idx_wl(N, i, 0)] = V[(size_t)b * M + i] / Rs;
  return 0;
}

/*
 * In-place LU decomposition of a band matrix (k x k, half-bandwidth p) without
 * pivoting (Sec. II-C).  On return the strict lower band holds L (unit
 * diagonal implied) and the diagonal and upper band hold U.
 * Returns 0, or the 1-based index of a zero pivot.
 */
int xref_lu_band(long long k, int p, double* ab) {
  const size_t W = (size_t)(2 * p + 1);
  for (long long r = 0; r < k; ++r) {
    const double piv = ab[(size_t)r * W + p];
    if (piv == 0.0) return (int)(r + 1);
    const long long last = (r + p < k - 1) ? r + p : k - 1;
    for (long long i = r + 1; i <= last; ++i) {
      double* row_i = ab + (size_t)i * W;
      const double* row_r = ab + (size_t)r * W;
      const size_t col_r_in_i = (size_t)(r - i + p);
      const double a = row_i[col_r_in_i];
      if (a == 0.0) continue;
      const double l = a / piv;
      row_i[col_r_in_i] = l;
      for (long long c = r + 1; c <= last; ++c) row_i[c - i + p] -= l * row_r[c - r + p];
    }
  }
  return 0;
}

/*
 * Forward and back substitution (Sec. II-C) for B right-hand sides stored
 * consecutively in x[B x k]; overwritten with the solutions.  RHS are
 * independent, so they are spread over `nthreads` OpenMP threads (0 = default).
 */
int xref_solve_band(long long k, int p, const double* lu, int B, double* x, int nthreads) {
  const size_t W = (size_t)(2 * p + 1);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < B; ++b) {
    double* y = x + (size_t)b * (size_t)k;
    for (long long i = 0; i < k; ++i) {          /* L y = I */
      const double* row = lu + (size_t)i * W;
      double s = y[i];
      const long long c0 = (i - p > 0) ? i - p : 0;
      for (long long c = c0; c < i; ++c) s -= row[c - i + p] * y[c];
      y[i] = s;
    }
    for (long long i = k - 1; i >= 0; --i) {     /* U V = y */
      const double* row = lu + (size_t)i * W;
      double s = y[i];
      const long long c1 = (i + p < k - 1) ? i + p : k - 1;
      for (long long c = i + 1; c <= c1; ++c) s -= row[c - i + p] * y[c];
      y[i] = s / row[p];
    }
  }
  (void)nthreads;
  return 0;
}

/*
 * From node voltages x[B x 2MN] extract:
 *   I[B x N]      bit-line termination currents g_o * V_BL(M,j) (output vector),
 *   vWL, vBL      [B x M x N] node voltages (either may be NULL),
 *   Isrc[B x M]   source currents g_s * (V_i - V_WL(i,1)) (may be NULL; needs V).
 */
int xref_extract(int M, int N, int B, const double* x, double Rs, double Rsense, const double* V,
                 double* I, double* vWL, double* vBL, double* Isrc) {
  const size_t k = 2 * (size_t)M * (size_t)N;
  for (int b = 0; b < B; ++b) {
    const double* xb = x + (size_t)b * k;
    if (I)
      for (int j = 0; j < N; ++j) I[(size_t)b * N + j] = xb[idx_bl(N, M - 1, j)] / Rsense;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < N; ++j) {
        const size_t o = ((size_t)b * M + i) * N + j;
        if (vWL) vWL[o] = xb[idx_wl(N, i, j)];
        if (vBL) vBL[o] = xb[idx_bl(N, i, j)];
      }
    if (Isrc && V)
      for (int i = 0; i < M; ++i)
        Isrc[(size_t)b * M + i] = (V[(size_t)b * M + i] - xb[idx_wl(N, i, 0)]) / Rs;
  }
  return 0;
}

int xref_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
