/* FP64 oracle: the global chemical potential of Eq. 2 by bisection on the collected count, in C.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only the tests, the smoke check and the CPU
 * baseline of the benchmark call it; the CUDA path never links it.
 *
 * One mu serves every subgraph (Sec. "Density Matrix Evaluation on Partitioned Graphs"), fixed by
 * the electron count collected from the core rows: N(mu) = 2 sum_i sum_k w_ik f(eps_ik - mu) = N_e,
 * with eps_ik the eigenvalues of subgraph i's orthogonalised Hamiltonian, w_ik the core Mulliken
 * weight of state k (oracle_subgraph_eig) and f the Fermi function at inverse temperature beta,
 * evaluated with the exponential of -|beta x| only.  The states of all subgraphs come as one
 * array; the count sums them in array order.
 */
#include <math.h>
#include <stdint.h>

static double fermi(double x, double beta) {
  const double e = exp(-fabs(beta * x));
  return x > 0.0 ? e / (1.0 + e) : 1.0 / (1.0 + e);
}

/* N(mu) over n states (eps, w: host arrays of n doubles). */
double oracle_collected_count(int64_t n, const double* eps, const double* w, double mu, double beta) {
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += w[k] * fermi(eps[k] - mu, beta);
  return 2.0 * s;
}

/* Bisection on N(mu) = n_e, N non-decreasing in mu.  Bracket [min eps - 1, max eps + 1]; stop when
 * |N - n_e| < 1e-11 or the bracket is narrower than 1e-15 Ha (at most 400 halvings); *mu receives
 * the midpoint.  Returns the number of halvings, -1 for n < 1 or a non-finite input. */
int oracle_solve_mu(int64_t n, const double* eps, const double* w, double n_e, double beta, double* mu) {
  if (n < 1 || !mu || !isfinite(n_e) || !(beta > 0.0)) return -1;
  double lo = eps[0], hi = eps[0];
  for (int64_t k = 0; k < n; ++k) {
    if (!isfinite(eps[k]) || !isfinite(w[k])) return -1;
    if (eps[k] < lo) lo = eps[k];
    if (eps[k] > hi) hi = eps[k];
  }
  lo -= 1.0;
  hi += 1.0;
  double mid = 0.5 * (lo + hi);
  int it = 0;
  for (; it < 400; ++it) {
    mid = 0.5 * (lo + hi);
    const double nel = oracle_collected_count(n, eps, w, mid, beta);
    if (fabs(nel - n_e) < 1e-11 || hi - lo < 1e-15) break;
    if (nel < n_e)
      lo = mid;
    else
      hi = mid;
  }
  *mu = mid;
  return it;
}
