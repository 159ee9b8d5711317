/*
 * ion_oracle.c -- plain FP64 CPU oracle for the multi-level ionization step of
 * Cheng & Samulyak, "Efficient numerical algorithm for multi-level ionization
 * of high-atomic-number gases" (arXiv 2202.10647).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * library; it is written to be slow and obviously correct.
 *
 * What it computes, per mesh cell c (Sec. 2 and Sec. 3 of the paper):
 *   1. W_k(E) for the charge states of the cell's window, from the ADK formula
 *      (Eq. 1) evaluated literally with pow/sqrt/exp and factorials in double.
 *   2. The window's rate matrix A (the [lo,hi] block of the bidiagonal matrix of
 *      Eq. 3, rates frozen over the step as stated just below Eq. 3), with the
 *      top state of the window absorbing (the reduced system of Eqs. 6-9 has no
 *      loss term on its last level).
 *   3. N'(window) = exp(dt A) N(window).  The analytic solution of Eqs. 4-5 (and
 *      its 4-level instance, Eqs. 6-9) is exactly this matrix exponential applied
 *      to the initial populations; the oracle evaluates the definition directly
 *      by scaling and squaring of the Taylor series (Moler & Van Loan,
 *      "Nineteen dubious ways", method 3), recomputing the diagonal exactly after
 *      every squaring as in Al-Mohy & Higham (SIMAX 2009, Sec. 2) so that stiff
 *      windows keep full accuracy.  This needs no distinct-eigenvalue
 *      assumption, so equal rates (the defective case Eq. 4 cannot express)
 *      are handled by the same code.
 *   4. dn_e = sum_k k (N'_k - N_k) over the window, times n_gas if given.
 *   5. The window slides up (lo++, hi++) while the new population of its lowest
 *      level is below eps_shift (Sec. 3, text after Fig. 2 and after Eq. 9),
 *      at most w-1 times and only while hi < Z.
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   - Q = k+1 for the rate W_k of state k -> k+1 ("charge number after
 *     ionization", text after Eq. 1).
 *   - E_L is the magnitude |E| given per cell; Eq. 1 is applied as printed
 *     (with its cycle-averaging square-root factor).
 *   - W = 0 when |E| <= 1e-6 GV/m or when the exponent (2/3)(Q/n*)^3 E_a/E
 *     exceeds 700 (the direct formula would form 0*inf there).
 *   - The constants default to the printed omega_a = 4.13e16 1/s, E_a = 510
 *     GV/m, and U_H = 13.6 eV (U_H is not printed).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXW 64 /* largest window the oracle accepts (Z+1 for Z <= 63) */

/* ------------------------------------------------------------------------- */
/* Eq. 1: the (l,|m|) factor (2l+1)(l+|m|)! / (2^|m| |m|! (l-|m|)!)           */
/* ------------------------------------------------------------------------- */
static double or_factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

double or_flm(int l, int m) {
  int am = m < 0 ? -m : m;
  return (2.0 * l + 1.0) * or_factorial(l + am) /
         (pow(2.0, (double)am) * or_factorial(am) * or_factorial(l - am));
}

/* ------------------------------------------------------------------------- */
/* Eq. 1: ADK rate in 1/fs for one transition.                               */
/*   E_GVm  : local field magnitude, GV/m                                    */
/*   U_eV   : ionization potential of the state being ionized, eV            */
/*   l, m   : orbital quantum number and its projection                      */
/*   Q      : charge number after ionization                                 */
/*   consts : {omega_a [1/s], E_a [GV/m], U_H [eV], model}                   */
/*            model 0: Eq. 1 as printed (cycle-averaged);                    */
/*            model 1: the static-field rate, Eq. 1 without the factor       */
/*            sqrt(3 n*^3 E / (pi Q^3 E_a)) that averages over a cycle.      */
/* ------------------------------------------------------------------------- */
double or_adk_rate(double E_GVm, double U_eV, int l, int m, int Q,
                   const double *consts) {
  const double omega_a = consts[0];
  const double E_a = consts[1];
  const double U_H = consts[2];
  const int model = (int)consts[3];
  const double E = fabs(E_GVm);
  const int am = m < 0 ? -m : m;
  const double q = (double)Q;
  const double nstar = q * sqrt(U_H / U_eV);
  if (!(E > 1e-6)) return 0.0;
  const double expo = (2.0 * E_a / (3.0 * E)) * pow(q / nstar, 3.0);
  if (expo > 700.0) return 0.0;
  const double e = exp(1.0);
  const double cycle =
      model == 1 ? 1.0 : sqrt(3.0 * pow(nstar, 3.0) * E / (M_PI * pow(q, 3.0) * E_a));
  const double W =
      omega_a * cycle *
      (q * q) / (2.0 * nstar * nstar) * pow(2.0 * e / nstar, 2.0 * nstar) *
      exp(-expo) *
      ((2.0 * l + 1.0) * or_factorial(l + am)) /
          (2.0 * M_PI * nstar * pow(2.0, (double)am) * or_factorial(am) *
           or_factorial(l - am)) *
      pow(2.0 * E_a * pow(q, 3.0) / (E * pow(nstar, 3.0)),
          2.0 * nstar - (double)am - 1.0);
  return W * 1e-15; /* 1/s -> 1/fs */
}

/* ------------------------------------------------------------------------- */
/* Dense n x n helpers (row-major), plain loops.                             */
/* ------------------------------------------------------------------------- */
static void mat_mul(int n, const double *A, const double *B, double *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

static double mat_norm_inf(int n, const double *A) {
  double mx = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fabs(A[i * n + j]);
    if (s > mx) mx = s;
  }
  return mx;
}

/* exp(M) for an n x n matrix M (row-major): scaling and squaring of the
 * Taylor series; if the matrix is lower triangular the diagonal is reset to the
 * exact exp(2^(i-s) M_jj) after squaring i (Al-Mohy & Higham 2009). */
void or_expm(int n, const double *M, double *X) {
  double B[OR_MAXW * OR_MAXW], T[OR_MAXW * OR_MAXW], U[OR_MAXW * OR_MAXW];
  int lower = 1;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (M[i * n + j] != 0.0) lower = 0;
  double nrm = mat_norm_inf(n, M);
  int s = 0;
  while (nrm > 0.5) {
    nrm *= 0.5;
    ++s;
  }
  const double scale = ldexp(1.0, -s);
  for (int i = 0; i < n * n; ++i) B[i] = M[i] * scale;
  /* X = sum_k B^k / k! */
  for (int i = 0; i < n * n; ++i) {
    X[i] = 0.0;
    T[i] = 0.0;
  }
  for (int i = 0; i < n; ++i) {
    X[i * n + i] = 1.0;
    T[i * n + i] = 1.0;
  }
  /* ||B|| <= 1/2: 30 terms beyond the nilpotent degree n-1 leave a remainder
   * below 2^-30/30! relative to every entry's leading term. */
  for (int k = 1; k <= n + 30; ++k) {
    mat_mul(n, T, B, U);
    for (int i = 0; i < n * n; ++i) {
      T[i] = U[i] / (double)k;
      X[i] += T[i];
    }
  }
  if (lower)
    for (int i = 0; i < n; ++i) X[i * n + i] = exp(B[i * n + i]);
  for (int r = 1; r <= s; ++r) {
    mat_mul(n, X, X, U);
    memcpy(X, U, sizeof(double) * n * n);
    if (lower)
      for (int i = 0; i < n; ++i) X[i * n + i] = exp(ldexp(B[i * n + i], r));
  }
}

/* ------------------------------------------------------------------------- */
/* Rates of states k_lo .. k_hi-1 for every cell (SoA out, [k][ncells]).     */
/* ------------------------------------------------------------------------- */
int or_rates(int Z, const double *U, const int *l, const int *m,
             const double *consts, int64_t ncells, const double *E, int k_lo,
             int k_hi, double *W_out, int nthreads) {
  if (Z < 1 || Z >= OR_MAXW || k_lo < 0 || k_hi > Z || k_lo > k_hi) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < ncells; ++c)
    for (int k = k_lo; k < k_hi; ++k)
      W_out[(int64_t)(k - k_lo) * ncells + c] =
          or_adk_rate(E[c], U[k], l[k], m[k], k + 1, consts);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One step of the windowed analytic update for every cell.                  */
/*   N      : SoA populations, plane k at N + k*ld, (Z+1) planes; in/out     */
/*   lo, hi : window bounds per cell; in/out                                 */
/*   dne    : out, newly freed electrons per cell (x n_gas if non-null)      */
/*   window_update : 0 keeps the windows fixed                               */
/*   policy : 0 the paper's rule (Sec. 3): slide up while the lowest state   */
/*            holds less than eps_shift, width kept;                         */
/*            1 adaptive: while the lowest state holds less than eps_shift,  */
/*            drop it if the width exceeds wmin, else slide; then, if the    */
/*            old top state holds more than eps_grow, add the state above    */
/*            (width at most wmax).                                          */
/* ------------------------------------------------------------------------- */
int or_step(int Z, const double *U, const int *l, const int *m,
            const double *consts, int64_t ncells, const double *E, double *N,
            int64_t ld, double dt, uint8_t *lo, uint8_t *hi, double *dne,
            const double *n_gas, double eps_shift, int window_update,
            int policy, int wmin, int wmax, double eps_grow, int nthreads) {
  if (Z < 1 || Z >= OR_MAXW || ld < ncells || dt < 0.0) return -1;
  for (int64_t c = 0; c < ncells; ++c)
    if (lo[c] > hi[c] || hi[c] > Z) return -2;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (int64_t c = 0; c < ncells; ++c) {
    const int a = lo[c], b = hi[c], w = b - a + 1;
    double A[OR_MAXW * OR_MAXW], P[OR_MAXW * OR_MAXW];
    double n0[OR_MAXW], n1[OR_MAXW];
    for (int i = 0; i < w * w; ++i) A[i] = 0.0;
    /* Eq. 3 restricted to the window; the top state has no outflow. */
    for (int i = 0; i < w - 1; ++i) {
      const int k = a + i;
      const double Wk = or_adk_rate(E[c], U[k], l[k], m[k], k + 1, consts);
      A[i * w + i] = -Wk * dt;
      A[(i + 1) * w + i] = Wk * dt;
    }
    or_expm(w, A, P);
    for (int i = 0; i < w; ++i) n0[i] = N[(int64_t)(a + i) * ld + c];
    for (int i = 0; i < w; ++i) {
      double s = 0.0;
      for (int j = 0; j < w; ++j) s += P[i * w + j] * n0[j];
      n1[i] = s;
    }
    double d = 0.0;
    for (int i = 0; i < w; ++i) d += (double)(a + i) * (n1[i] - n0[i]);
    dne[c] = n_gas ? d * n_gas[c] : d;
    for (int i = 0; i < w; ++i) N[(int64_t)(a + i) * ld + c] = n1[i];
    if (window_update && policy == 0) {
      int na = a, nb = b, shifts = 0;
      while (shifts < w - 1 && nb < Z && N[(int64_t)na * ld + c] < eps_shift) {
        ++na;
        ++nb;
        ++shifts;
      }
      lo[c] = (uint8_t)na;
      hi[c] = (uint8_t)nb;
    } else if (window_update) {
      int na = a, nb = b;
      for (int moves = 0; moves < w - 1; ++moves) {
        if (!(N[(int64_t)na * ld + c] < eps_shift)) break;
        if (nb - na + 1 > wmin) {
          ++na;
        } else if (nb < Z) {
          ++na;
          ++nb;
        } else {
          break;
        }
      }
      if (N[(int64_t)b * ld + c] > eps_grow && nb < Z && nb - na + 1 < wmax) ++nb;
      lo[c] = (uint8_t)na;
      hi[c] = (uint8_t)nb;
    }
  }
  return 0;
}

/* Number of threads OpenMP would use (for reporting the CPU baseline). */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
