/*
 * Plain CPU oracle for the sector-restricted Fock-space evolution of
 * Eberhardt, Zamora, Kopp & Abel, "On the single classical field description
 * of interacting scalar fields" (arXiv:2111.00050).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything here is written for obviousness, not speed:
 *   - a sector basis is every composition of N into M parts whose momentum is
 *     P (mod M), enumerated by brute force in lexicographic order (Sec. III B,
 *     "special Hilbert spaces");
 *   - the Hamiltonian (Eq. Ham, with L_{pq;rs} = Lambda^{rs}_{pq}/2) is applied
 *     by literally acting with a_s, a_r, a_q^dag, a_p^dag on each basis ket for
 *     every ordered tuple (p,q,r,s), and the resulting ket is located by binary
 *     search in the sorted basis;
 *   - time stepping is the classic four-stage Runge-Kutta scheme;
 *   - moments <a_i>, <a_i^dag a_j>, <a_i a_j> are accumulated by acting with the
 *     operators on every ket of the concatenated multi-sector state (Sec. II C-E).
 *
 * Complex numbers are stored as interleaved (re, im) doubles.
 * Mode labels: for odd M, mode index i carries momentum label i - (M-1)/2; for
 * even M the label is i.  Momentum is conserved modulo M, or exactly (the plain
 * label sum, Sec. III B) where a function takes exact = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int label_of(int M, int i) { return (M % 2) ? i - (M - 1) / 2 : i; }

static int mod_pos(int a, int M) {
  int r = a % M;
  return r < 0 ? r + M : r;
}

/* the mode index s whose label is congruent to k (mod M); unique for both label
 * conventions */
static int mode_of_residue(int M, int k) {
  for (int i = 0; i < M; ++i)
    if (mod_pos(label_of(M, i) - k, M) == 0) return i;
  return -1;
}

/* total momentum of a ket: the label sum, reduced mod M unless exact */
static int momentum_of(int M, const int* n, int exact) {
  int k = 0;
  for (int i = 0; i < M; ++i) k += label_of(M, i) * n[i];
  return exact ? k : mod_pos(k, M);
}

/* a momentum label sum, reduced mod M unless exact */
static int pwrap(int k, int M, int exact) { return exact ? k : mod_pos(k, M); }

/* ---- basis enumeration (Sec. III B: the special Hilbert space of (N, P)) ---- */

static void enum_rec(int M, int m, int rem, int P, int exact, int* cur, int64_t* count, int* out, int64_t cap) {
  if (m == M - 1) {
    cur[m] = rem;
    if (momentum_of(M, cur, exact) == P) {
      if (out && *count < cap) memcpy(out + (*count) * M, cur, sizeof(int) * (size_t)M);
      ++*count;
    }
    return;
  }
  for (int v = 0; v <= rem; ++v) {
    cur[m] = v;
    enum_rec(M, m + 1, rem - v, P, exact, cur, count, out, cap);
  }
}

/* Number of kets with sum n = N and momentum P (mod M, or exactly); if out !=
 * NULL the first `cap` occupation vectors are written row-major [count][M] in
 * lexicographic order (n_0 ascending, then n_1, ...).  Returns the total count. */
int64_t orc_sector_basis(int M, int N, int P, int exact, int* out, int64_t cap) {
  int cur[64];
  int64_t count = 0;
  if (M < 1 || M > 64 || N < 0) return -1;
  enum_rec(M, 0, N, pwrap(P, M, exact), exact, cur, &count, out, cap);
  return count;
}

/* lexicographic comparison of two occupation vectors */
static int cmp_occ(int M, const int* a, const int* b) {
  for (int i = 0; i < M; ++i) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}

/* index of `occ` in the sorted basis [D][M], or -1 */
static int64_t find_ket(int M, const int* basis, int64_t D, const int* occ) {
  int64_t lo = 0, hi = D - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int c = cmp_occ(M, basis + mid * M, occ);
    if (c == 0) return mid;
    if (c < 0)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

int64_t orc_find(int M, const int* basis, int64_t D, const int* occ) { return find_ket(M, basis, D, occ); }

/* Rejects a coupling tensor with a nonzero entry on a tuple that does not
 * conserve momentum (mod M, or exactly; the delta in Eq. Lambda).  Returns 0 if
 * valid. */
int orc_check_coupling(int M, const double* L, int exact) {
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s) {
          int64_t t = (((int64_t)p * M + q) * M + r) * M + s;
          int cons = pwrap(label_of(M, p) + label_of(M, q) - label_of(M, r) - label_of(M, s), M, exact) == 0;
          if (!cons && (L[2 * t] != 0.0 || L[2 * t + 1] != 0.0)) return -1;
        }
  return 0;
}

/*
 * out = H psi (dagger = 0) or out = H^dag psi (dagger = 1) within one sector.
 * H = sum_p w_p a_p^dag a_p + sum_{p,q,r,s} L_{pq;rs} a_p^dag a_q^dag a_r a_s
 * (Eq. Ham with L = Lambda/2), all ordered tuples, L complex [M^4] indexed
 * ((p*M+q)*M+r)*M+s.  Push form: each ket j is acted on and its amplitude is
 * added to the ket it lands on.  Returns 0, or -1 if some term leaves the basis.
 */
int orc_apply_h(int M, int64_t D, const int* basis, const double* w, const double* L, const double* psi,
                double* out, int dagger) {
  int tmp[64], r2m[64];
  for (int k = 0; k < M; ++k) r2m[k] = mode_of_residue(M, k);
  memset(out, 0, sizeof(double) * 2 * (size_t)D);
  for (int64_t j = 0; j < D; ++j) {
    const int* n = basis + j * M;
    double pr = psi[2 * j], pi = psi[2 * j + 1];
    /* one-body part: w_p a_p^dag a_p is diagonal */
    double diag = 0.0;
    for (int p = 0; p < M; ++p) diag += w[p] * n[p];
    out[2 * j] += diag * pr;
    out[2 * j + 1] += diag * pi;
    /* two-body part: every ordered tuple (p,q,r,s); momentum conservation mod M
     * (the Kronecker delta of Eq. Lambda) leaves one s for each (p,q,r) */
    for (int p = 0; p < M; ++p)
      for (int q = 0; q < M; ++q)
        for (int r = 0; r < M; ++r) {
          int s = r2m[mod_pos(label_of(M, p) + label_of(M, q) - label_of(M, r), M)];
            int64_t t = (((int64_t)p * M + q) * M + r) * M + s;
            double lr = L[2 * t], li = L[2 * t + 1];
            if (lr == 0.0 && li == 0.0) continue;
            memcpy(tmp, n, sizeof(int) * (size_t)M);
            double coef = 1.0;
            /* a_s */
            if (tmp[s] == 0) continue;
            coef *= sqrt((double)tmp[s]);
            tmp[s] -= 1;
            /* a_r */
            if (tmp[r] == 0) continue;
            coef *= sqrt((double)tmp[r]);
            tmp[r] -= 1;
            /* a_q^dag */
            tmp[q] += 1;
            coef *= sqrt((double)tmp[q]);
            /* a_p^dag */
            tmp[p] += 1;
            coef *= sqrt((double)tmp[p]);
            int64_t i = find_ket(M, basis, D, tmp);
            if (i < 0) return -1;
            double cr = lr * coef, ci = li * coef; /* <n_i| term |n_j> */
            if (!dagger) {
              out[2 * i] += cr * pr - ci * pi;
              out[2 * i + 1] += cr * pi + ci * pr;
            } else {
              double qr = psi[2 * i], qi = psi[2 * i + 1];
              out[2 * j] += cr * qr + ci * qi; /* conj(c) * psi_i */
              out[2 * j + 1] += cr * qi - ci * qr;
            }
          }
  }
  return 0;
}

/* f = -i H v */
static int deriv(int M, int64_t D, const int* basis, const double* w, const double* L, const double* v, double* f) {
  int rc = orc_apply_h(M, D, basis, w, L, v, f, 0);
  for (int64_t k = 0; k < D; ++k) {
    double hr = f[2 * k], hi = f[2 * k + 1];
    f[2 * k] = hi;
    f[2 * k + 1] = -hr;
  }
  return rc;
}

/*
 * Classic four-stage Runge-Kutta for d psi/dt = -i H psi (Eq. Schr) on one
 * sector, `steps` steps of size dt, in place.  Returns 0 or -1.
 */
int orc_rk4(int M, int64_t D, const int* basis, const double* w, const double* L, double* psi, double dt,
            int64_t steps) {
  size_t bytes = sizeof(double) * 2 * (size_t)D;
  double* k1 = malloc(bytes);
  double* k2 = malloc(bytes);
  double* k3 = malloc(bytes);
  double* k4 = malloc(bytes);
  double* u = malloc(bytes);
  int rc = 0;
  if (!k1 || !k2 || !k3 || !k4 || !u) rc = -2;
  for (int64_t st = 0; st < steps && rc == 0; ++st) {
    rc |= deriv(M, D, basis, w, L, psi, k1);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + 0.5 * dt * k1[k];
    rc |= deriv(M, D, basis, w, L, u, k2);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + 0.5 * dt * k2[k];
    rc |= deriv(M, D, basis, w, L, u, k3);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + dt * k3[k];
    rc |= deriv(M, D, basis, w, L, u, k4);
    for (int64_t k = 0; k < 2 * D; ++k) psi[k] += dt / 6.0 * (k1[k] + 2.0 * k2[k] + 2.0 * k3[k] + k4[k]);
  }
  free(k1);
  free(k2);
  free(k3);
  free(k4);
  free(u);
  return rc;
}

/* sector index holding (N, P), or -1 */
static int find_sector(int nsec, const int* secN, const int* secP, int N, int P) {
  for (int s = 0; s < nsec; ++s)
    if (secN[s] == N && secP[s] == P) return s;
  return -1;
}

/*
 * Raw (unnormalised) moments of a multi-sector state (Sec. II C-E):
 *   out[0]            = <psi|psi>
 *   out[1]            = <psi|N|psi>
 *   out[2 .. 2+2M)    = <psi|a_i|psi>            (complex, i = 0..M-1)
 *   next 2M^2         = <psi|a_i^dag a_j|psi>     (complex, row-major i, j)
 *   next 2M^2         = <psi|a_i a_j|psi>         (complex, row-major i, j)
 * Sector s holds kets basis[off[s] .. off[s+1]) of (secN[s], secP[s]); psi is
 * concatenated in the same order.  A ket an operator maps outside the held
 * sectors contributes zero (truncated space).
 */
void orc_moments(int M, int nsec, const int* secN, const int* secP, const int64_t* off, const int* basis,
                 const double* psi, double* out, int exact) {
  int tmp[64];
  int nout = 2 + 2 * M + 4 * M * M;
  memset(out, 0, sizeof(double) * (size_t)nout);
  double* A = out + 2;
  double* Mm = A + 2 * M;
  double* AA = Mm + 2 * M * M;
  for (int s = 0; s < nsec; ++s) {
    for (int64_t j = off[s]; j < off[s + 1]; ++j) {
      const int* n = basis + j * M;
      double pr = psi[2 * j], pi = psi[2 * j + 1];
      double p2 = pr * pr + pi * pi;
      int Ntot = 0;
      for (int i = 0; i < M; ++i) Ntot += n[i];
      out[0] += p2;
      out[1] += p2 * Ntot;
      /* <a_i>: a_i |n> = sqrt(n_i) |n - e_i> */
      for (int i = 0; i < M; ++i) {
        if (n[i] == 0) continue;
        memcpy(tmp, n, sizeof(int) * (size_t)M);
        double c = sqrt((double)tmp[i]);
        tmp[i] -= 1;
        int t = find_sector(nsec, secN, secP, secN[s] - 1, pwrap(secP[s] - label_of(M, i), M, exact));
        if (t < 0) continue;
        int64_t k = find_ket(M, basis + off[t] * M, off[t + 1] - off[t], tmp);
        if (k < 0) continue;
        k += off[t];
        double qr = psi[2 * k], qi = psi[2 * k + 1];
        /* conj(psi_k) * c * psi_j */
        A[2 * i] += c * (qr * pr + qi * pi);
        A[2 * i + 1] += c * (qr * pi - qi * pr);
      }
      /* <a_i^dag a_j> */
      for (int i = 0; i < M; ++i)
        for (int jj = 0; jj < M; ++jj) {
          if (n[jj] == 0) continue;
          memcpy(tmp, n, sizeof(int) * (size_t)M);
          double c = sqrt((double)tmp[jj]);
          tmp[jj] -= 1;
          tmp[i] += 1;
          c *= sqrt((double)tmp[i]);
          int t = find_sector(nsec, secN, secP, secN[s], pwrap(secP[s] - label_of(M, jj) + label_of(M, i), M, exact));
          if (t < 0) continue;
          int64_t k = find_ket(M, basis + off[t] * M, off[t + 1] - off[t], tmp);
          if (k < 0) continue;
          k += off[t];
          double qr = psi[2 * k], qi = psi[2 * k + 1];
          Mm[2 * (i * M + jj)] += c * (qr * pr + qi * pi);
          Mm[2 * (i * M + jj) + 1] += c * (qr * pi - qi * pr);
        }
      /* <a_i a_j> */
      for (int i = 0; i < M; ++i)
        for (int jj = 0; jj < M; ++jj) {
          if (n[jj] == 0) continue;
          memcpy(tmp, n, sizeof(int) * (size_t)M);
          double c = sqrt((double)tmp[jj]);
          tmp[jj] -= 1;
          if (tmp[i] == 0) continue;
          c *= sqrt((double)tmp[i]);
          tmp[i] -= 1;
          int t = find_sector(nsec, secN, secP, secN[s] - 2,
                              pwrap(secP[s] - label_of(M, jj) - label_of(M, i), M, exact));
          if (t < 0) continue;
          int64_t k = find_ket(M, basis + off[t] * M, off[t + 1] - off[t], tmp);
          if (k < 0) continue;
          k += off[t];
          double qr = psi[2 * k], qi = psi[2 * k + 1];
          AA[2 * (i * M + jj)] += c * (qr * pr + qi * pi);
          AA[2 * (i * M + jj) + 1] += c * (qr * pi - qi * pr);
        }
    }
  }
}

/*
 * out = O psi for a single-mode operator O in {a_i (kind 0), a_i^dag (kind 1),
 * n_i (kind 2)} on a multi-sector state (targets outside the held sectors are
 * dropped).  Used to form gradients of moment-based losses.
 */
void orc_apply_mode_op(int M, int nsec, const int* secN, const int* secP, const int64_t* off, const int* basis,
                       const double* psi, int kind, int i, double* out, int exact) {
  int tmp[64];
  memset(out, 0, sizeof(double) * 2 * (size_t)off[nsec]);
  for (int s = 0; s < nsec; ++s) {
    for (int64_t j = off[s]; j < off[s + 1]; ++j) {
      const int* n = basis + j * M;
      double pr = psi[2 * j], pi = psi[2 * j + 1];
      memcpy(tmp, n, sizeof(int) * (size_t)M);
      double c;
      int tN, tP;
      if (kind == 2) {
        out[2 * j] += n[i] * pr;
        out[2 * j + 1] += n[i] * pi;
        continue;
      } else if (kind == 0) {
        if (tmp[i] == 0) continue;
        c = sqrt((double)tmp[i]);
        tmp[i] -= 1;
        tN = secN[s] - 1;
        tP = pwrap(secP[s] - label_of(M, i), M, exact);
      } else {
        tmp[i] += 1;
        c = sqrt((double)tmp[i]);
        tN = secN[s] + 1;
        tP = pwrap(secP[s] + label_of(M, i), M, exact);
      }
      int t = find_sector(nsec, secN, secP, tN, tP);
      if (t < 0) continue;
      int64_t k = find_ket(M, basis + off[t] * M, off[t + 1] - off[t], tmp);
      if (k < 0) continue;
      k += off[t];
      out[2 * k] += c * pr;
      out[2 * k + 1] += c * pi;
    }
  }
}

/*
 * (H psi)_i for the single ket i of one sector, by definition:
 * (H psi)_i = sum_j <n_i|H|n_j> psi_j, and <n_i|H|n_j> = conj(<n_j|H^dag|n_i>),
 * where H^dag = sum_p w_p n_p + sum conj(L_{pq;rs}) a_s^dag a_r^dag a_q a_p is
 * applied literally to |n_i>.  Lets a test check sampled rows of a sector far
 * too large for the push-form orc_apply_h.  Returns 0 or -1.
 */
int orc_apply_h_row(int M, int64_t D, const int* basis, const double* w, const double* L, const double* psi,
                    int64_t i, double* out2) {
  int tmp[64];
  const int* n = basis + i * M;
  double accr = 0.0, acci = 0.0;
  double diag = 0.0;
  for (int p = 0; p < M; ++p) diag += w[p] * n[p];
  accr += diag * psi[2 * i];
  acci += diag * psi[2 * i + 1];
  int r2m[64];
  for (int k = 0; k < M; ++k) r2m[k] = mode_of_residue(M, k);
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r) {
        int s = r2m[mod_pos(label_of(M, p) + label_of(M, q) - label_of(M, r), M)];
          int64_t t = (((int64_t)p * M + q) * M + r) * M + s;
          double lr = L[2 * t], li = L[2 * t + 1];
          if (lr == 0.0 && li == 0.0) continue;
          memcpy(tmp, n, sizeof(int) * (size_t)M);
          double coef = 1.0;
          /* adjoint term conj(L) a_s^dag a_r^dag a_q a_p: a_p first */
          if (tmp[p] == 0) continue;
          coef *= sqrt((double)tmp[p]);
          tmp[p] -= 1;
          if (tmp[q] == 0) continue;
          coef *= sqrt((double)tmp[q]);
          tmp[q] -= 1;
          tmp[r] += 1;
          coef *= sqrt((double)tmp[r]);
          tmp[s] += 1;
          coef *= sqrt((double)tmp[s]);
          int64_t j = find_ket(M, basis, D, tmp);
          if (j < 0) return -1;
          /* <n_j|H^dag|n_i> = conj(L) coef; <n_i|H|n_j> = L coef */
          double cr = lr * coef, ci = li * coef;
          double xr = psi[2 * j], xi = psi[2 * j + 1];
          accr += cr * xr - ci * xi;
          acci += cr * xi + ci * xr;
        }
  out2[0] = accr;
  out2[1] = acci;
  return 0;
}

/*
 * Number of distinct nonzero matrix elements <n_i|H|n_j> over all columns j of
 * one sector, diagonal included (structural count: every ket a term reaches
 * with a nonzero coupling counts once per column).  Used to express the
 * oracle's speed in H psi terms per second.
 */
int64_t orc_count_terms(int M, int64_t D, const int* basis, const double* L) {
  int tmp[64], r2m[64];
  for (int k = 0; k < M; ++k) r2m[k] = mode_of_residue(M, k);
  int64_t total = 0;
  int64_t cap = 1024, *tg = malloc(sizeof(int64_t) * (size_t)cap);
  for (int64_t j = 0; j < D; ++j) {
    const int* n = basis + j * M;
    int64_t nt = 0;
    tg[nt++] = j; /* the diagonal */
    for (int p = 0; p < M; ++p)
      for (int q = 0; q < M; ++q)
        for (int r = 0; r < M; ++r) {
          int s = r2m[mod_pos(label_of(M, p) + label_of(M, q) - label_of(M, r), M)];
            int64_t t = (((int64_t)p * M + q) * M + r) * M + s;
            if (L[2 * t] == 0.0 && L[2 * t + 1] == 0.0) continue;
            memcpy(tmp, n, sizeof(int) * (size_t)M);
            if (tmp[s] == 0) continue;
            tmp[s] -= 1;
            if (tmp[r] == 0) continue;
            tmp[r] -= 1;
            tmp[q] += 1;
            tmp[p] += 1;
            int64_t i = find_ket(M, basis, D, tmp);
            if (i < 0) continue;
            int seen = 0;
            for (int64_t k = 0; k < nt; ++k)
              if (tg[k] == i) seen = 1;
            if (!seen) {
              if (nt == cap) {
                cap *= 2;
                tg = realloc(tg, sizeof(int64_t) * (size_t)cap);
              }
              tg[nt++] = i;
            }
          }
    total += nt;
  }
  free(tg);
  return total;
}

/* f = -i H v row by row (orc_apply_h_row, the pull form, which the tests pin to
   the push form).  The rows are independent: a build with OpenMP (-fopenmp) runs
   them on every host core, which is the timed CPU baseline; without it this is the
   same loop on one core. */
static int deriv_rows(int M, int64_t D, const int* basis, const double* w, const double* L, const double* v,
                      double* f) {
  int rc = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(| : rc)
#endif
  for (int64_t i = 0; i < D; ++i) {
    double h[2];
    rc |= orc_apply_h_row(M, D, basis, w, L, v, i, h);
    f[2 * i] = h[1];
    f[2 * i + 1] = -h[0];
  }
  return rc;
}

/* orc_rk4 with H psi formed row by row (deriv_rows). */
int orc_rk4_rows(int M, int64_t D, const int* basis, const double* w, const double* L, double* psi, double dt,
                 int64_t steps) {
  size_t bytes = sizeof(double) * 2 * (size_t)D;
  double* k1 = malloc(bytes);
  double* k2 = malloc(bytes);
  double* k3 = malloc(bytes);
  double* k4 = malloc(bytes);
  double* u = malloc(bytes);
  int rc = 0;
  if (!k1 || !k2 || !k3 || !k4 || !u) rc = -2;
  for (int64_t st = 0; st < steps && rc == 0; ++st) {
    rc |= deriv_rows(M, D, basis, w, L, psi, k1);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + 0.5 * dt * k1[k];
    rc |= deriv_rows(M, D, basis, w, L, u, k2);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + 0.5 * dt * k2[k];
    rc |= deriv_rows(M, D, basis, w, L, u, k3);
    for (int64_t k = 0; k < 2 * D; ++k) u[k] = psi[k] + dt * k3[k];
    rc |= deriv_rows(M, D, basis, w, L, u, k4);
    for (int64_t k = 0; k < 2 * D; ++k) psi[k] += dt / 6.0 * (k1[k] + 2.0 * k2[k] + 2.0 * k3[k] + k4[k]);
  }
  free(k1);
  free(k2);
  free(k3);
  free(k4);
  free(u);
  return rc;
}

/* threads a parallel region of this build uses (1 without OpenMP) */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
