/* FP64 oracle: the per-subgraph eigensolve by cyclic Jacobi rotations, in plain C.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only the tests, the smoke check and the CPU
 * baseline of the benchmark call it; the CUDA path never links it.
 *
 * What it computes, for one core+halo subgraph with Hamiltonian block h and overlap block s (both
 * n x n, symmetric, row-major), in the order of the paper's subgraph solve (Sec. "Density Matrix
 * Evaluation on Partitioned Graphs": change to an orthonormal basis, then the Fermi operator of the
 * orthogonalised Hamiltonian through its eigen-decomposition):
 *   1. s = U diag(lam) U^T                          (Jacobi)
 *   2. Z = U diag(lam^-1/2) U^T = s^-1/2
 *   3. h~ = Z h Z, symmetrised as (h~ + h~^T) / 2
 *   4. h~ = X diag(eps) X^T                         (Jacobi), eps ascending
 *   5. C = Z X (the states in the atomic-orbital basis)
 *   6. w_k = sum_{i < n_core_orb} C_ik (s C)_ik      (core Mulliken weight of state k)
 * The occupations, the chemical potential (bisection on the collected count, Eq. 2) and the
 * collected observables stay in the Python oracle, which calls this for the eigenpairs.
 *
 * The eigensolver is the classical cyclic Jacobi method (C. G. J. Jacobi, 1846; row-cyclic sweeps
 * over the pairs p < q as in Golub and Van Loan, "Matrix Computations", Sec. 8.5).  Each rotation
 * J in the (p, q) plane makes B = J^T A J have B_pq = 0: with theta = (a_qq - a_pp) / (2 a_pq) the
 * tangent t = s / c is the root of t^2 + 2 theta t - 1 = 0 of smaller modulus,
 * t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1 / sqrt(1 + t^2), s = t c; then
 * B_pp = a_pp - t a_pq, B_qq = a_qq + t a_pq, and for r != p, q: B_rp = c a_rp - s a_rq,
 * B_rq = s a_rp + c a_rq.  The accumulated product of the rotations holds the eigenvectors.
 * Both updates are applied as small corrections, x' = x - s (y + tau x) and y' = y + s (x - tau y)
 * with tau = s / (1 + c) (the same values, since 1 - c = s tau; Rutishauser's form of the rotation,
 * which loses less to rounding when the rotations are small, as in the last sweeps).
 * Sweeps stop when the off-diagonal Frobenius norm is at most 1e-15 of the matrix's Frobenius norm
 * (quadratic convergence: a handful of sweeps); a sweep limit of 60 reports failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double off_norm2(int n, const double* a) {
  double s = 0.0;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) s += 2.0 * a[(int64_t)p * n + q] * a[(int64_t)p * n + q];
  return s;
}

/* Eigen-decomposition of the symmetric n x n matrix a (row-major, destroyed).  On return
 * w[0..n) holds the eigenvalues in ascending order and column k of v (row-major n x n) the unit
 * eigenvector of w[k].  work: n^2 + n doubles.  Returns the number of sweeps, -1 without
 * convergence within 60 sweeps, -2 for n < 0, -4 when out of memory. */
int oracle_jacobi_eigh(int n, double* a, double* v, double* w, double* work) {
  if (n < 0) return -2;
  if (n == 0) return 0;
  /* rows of vt are the eigenvectors while rotating (contiguous updates) */
  double* vt = work;
  double* tmp = work + (int64_t)n * n;
  memset(vt, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i) vt[(int64_t)i * n + i] = 1.0;
  double fro2 = 0.0;
  for (int64_t i = 0; i < (int64_t)n * n; ++i) fro2 += a[i] * a[i];
  const double stop2 = 1e-30 * fro2;
  int sweeps = 0;
  while (off_norm2(n, a) > stop2) {
    if (sweeps == 60) return -1;
    ++sweeps;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double* rp = a + (int64_t)p * n;
        double* rq = a + (int64_t)q * n;
        const double apq = rp[q];
        if (apq == 0.0) continue;
        const double theta = (rq[q] - rp[p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = t * c;
        const double tau = s / (1.0 + c);
        const double app = rp[p] - t * apq;
        const double aqq = rq[q] + t * apq;
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          const double arp = rp[r], arq = rq[r];
          const double bp = arp - s * (arq + tau * arp);
          const double bq = arq + s * (arp - tau * arq);
          rp[r] = bp;
          rq[r] = bq;
          a[(int64_t)r * n + p] = bp;
          a[(int64_t)r * n + q] = bq;
        }
        rp[p] = app;
        rq[q] = aqq;
        rp[q] = 0.0;
        rq[p] = 0.0;
        double* vp = vt + (int64_t)p * n;
        double* vq = vt + (int64_t)q * n;
        for (int k = 0; k < n; ++k) {
          const double x = vp[k], y = vq[k];
          vp[k] = x - s * (y + tau * x);
          vq[k] = y + s * (x - tau * y);
        }
      }
    }
  }
  /* ascending order: selection of the smallest remaining diagonal entry (ties keep index order) */
  for (int i = 0; i < n; ++i) w[i] = a[(int64_t)i * n + i];
  int* idx = (int*)malloc(sizeof(int) * (size_t)n);
  if (!idx) return -4;
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (w[idx[j]] < w[idx[m]]) m = j;
    const int t = idx[i];
    idx[i] = idx[m];
    idx[m] = t;
  }
  for (int k = 0; k < n; ++k) tmp[k] = w[idx[k]];
  memcpy(w, tmp, sizeof(double) * (size_t)n);
  for (int k = 0; k < n; ++k) {
    const double* src = vt + (int64_t)idx[k] * n;
    for (int i = 0; i < n; ++i) v[(int64_t)i * n + k] = src[i];
  }
  free(idx);
  return sweeps;
}

/* c = a b for n x n row-major matrices (plain triple loop, i-k-j order). */
static void matmul(int n, const double* a, const double* b, double* c) {
  memset(c, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double x = a[(int64_t)i * n + k];
      const double* bk = b + (int64_t)k * n;
      double* ci = c + (int64_t)i * n;
      for (int j = 0; j < n; ++j) ci[j] += x * bk[j];
    }
}

/* Steps 1-6 above for one subgraph.  h, s: n x n (row-major, read only).  Outputs: z (n x n),
 * eps (n), xv (n x n, the eigenvectors X of h~ in columns), cst (n x n, C = Z X), w (n).
 * Returns 0, or the negative status of the eigensolver (-1: no convergence), or -3 when s is not
 * positive definite, -4 when out of memory. */
int oracle_subgraph_eig(int n, int n_core_orb, const double* h, const double* s, double* z, double* eps,
                        double* xv, double* cst, double* w) {
  if (n < 0 || n_core_orb < 0 || n_core_orb > n) return -2;
  if (n == 0) return 0;
  const size_t nn = (size_t)n * n;
  double* buf = (double*)malloc(sizeof(double) * (6 * nn + 2 * (size_t)n));
  if (!buf) return -4;
  double* a = buf;
  double* u = a + nn;
  double* t = u + nn;
  double* x = t + nn;
  double* lam = x + nn;
  double* sc = lam + n;
  double* work = sc + nn;
  int st;
  memcpy(a, s, sizeof(double) * nn);
  if ((st = oracle_jacobi_eigh(n, a, u, lam, work)) < 0) { free(buf); return st; }
  for (int k = 0; k < n; ++k)
    if (!(lam[k] > 0.0)) { free(buf); return -3; }
  /* Z = U diag(lam^-1/2) U^T */
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) t[(int64_t)i * n + k] = u[(int64_t)i * n + k] / sqrt(lam[k]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += t[(int64_t)i * n + k] * u[(int64_t)j * n + k];
      z[(int64_t)i * n + j] = acc;
    }
  /* h~ = Z h Z, symmetrised */
  matmul(n, z, h, t);
  matmul(n, t, z, a);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double m = 0.5 * (a[(int64_t)i * n + j] + a[(int64_t)j * n + i]);
      a[(int64_t)i * n + j] = m;
      a[(int64_t)j * n + i] = m;
    }
  if ((st = oracle_jacobi_eigh(n, a, x, eps, work)) < 0) { free(buf); return st; }
  memcpy(xv, x, sizeof(double) * nn);
  matmul(n, z, x, cst);
  matmul(n, s, cst, sc);
  for (int k = 0; k < n; ++k) {
    double acc = 0.0;
    for (int i = 0; i < n_core_orb; ++i) acc += cst[(int64_t)i * n + k] * sc[(int64_t)i * n + k];
    w[k] = acc;
  }
  free(buf);
  return 0;
}

/* oracle_subgraph_eig over n_sub independent subgraphs, spread over the host's threads (OpenMP,
 * dynamic schedule, largest first is the caller's choice of order).  Subgraph i has size n[i],
 * core orbitals nco[i], its h, s, z, xv and cst at element offset sq_off[i] and its eps and w at
 * vec_off[i].  status[i] receives each subgraph's return value; returns 0 when all are 0, else
 * the first nonzero status in subgraph order. */
int oracle_subgraph_eig_batch(int n_sub, const int* n, const int* nco, const int64_t* sq_off,
                              const int64_t* vec_off, const double* h, const double* s, double* z,
                              double* eps, double* xv, double* cst, double* w, int* status) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n_sub; ++i)
    status[i] = oracle_subgraph_eig(n[i], nco[i], h + sq_off[i], s + sq_off[i], z + sq_off[i], eps + vec_off[i],
                                    xv + sq_off[i], cst + sq_off[i], w + vec_off[i]);
  for (int i = 0; i < n_sub; ++i)
    if (status[i] != 0) return status[i];
  return 0;
}
