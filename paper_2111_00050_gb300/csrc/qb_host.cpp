// Host side of the qb library: model validation, sector tables, the C ABI
// entry points, the small Hermitian eigensolve behind the Penrose-Onsager
// test, breaktime detection and the mean-field integrator.
//
// Paper: Eberhardt, Zamora, Kopp & Abel, arXiv:2111.00050.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "qb_internal.h"

namespace qb {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

typedef std::complex<double> cd;

static int label_shift(int M) { return (M % 2) ? (M - 1) / 2 : 0; }
static int modp(long long a, int M) {
  long long r = a % M;
  return (int)(r < 0 ? r + M : r);
}
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Validates and symmetrises the coupling tensor (see qb_model in qb.h).
static int prepare_model(const qb_model* model, std::vector<double>& w, std::vector<double>& Lsym) {
  if (!model || !model->w || !model->L) return fail(QB_EINVAL, "model, model->w and model->L must be non-NULL");
  const int M = model->M;
  if (M < 1 || M > QB_MAX_MODES) return fail(QB_EUNSUPPORTED, "M must be in [1, QB_MAX_MODES]");
  const int c = label_shift(M);
  w.assign(model->w, model->w + M);
  for (int p = 0; p < M; ++p)
    if (!std::isfinite(w[p])) return fail(QB_EINVAL, "w has a non-finite entry");
  const size_t M4 = (size_t)M * M * M * M;
  auto Lat = [&](int p, int q, int r, int s) {
    size_t t = (((size_t)p * M + q) * M + r) * M + s;
    return cd(model->L[2 * t], model->L[2 * t + 1]);
  };
  double lmax = 0.0;
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s) {
          cd v = Lat(p, q, r, s);
          if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return fail(QB_EINVAL, "L has a non-finite entry");
          lmax = std::max(lmax, std::abs(v));
          const long long dP = (long long)(p - c) + (q - c) - (r - c) - (s - c);
          bool cons = model->exact_momentum ? dP == 0 : modp(dP, M) == 0;
          if (!cons && v != cd(0, 0))
            return fail(QB_EINVAL, model->exact_momentum ? "L is nonzero on a tuple that does not conserve momentum"
                                                         : "L is nonzero on a tuple that does not conserve momentum mod M");
        }
  Lsym.assign(2 * M4, 0.0);
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s) {
          cd v = 0.25 * (Lat(p, q, r, s) + Lat(q, p, r, s) + Lat(p, q, s, r) + Lat(q, p, s, r));
          size_t t = (((size_t)p * M + q) * M + r) * M + s;
          Lsym[2 * t] = v.real();
          Lsym[2 * t + 1] = v.imag();
        }
  auto S = [&](int p, int q, int r, int s) {
    size_t t = (((size_t)p * M + q) * M + r) * M + s;
    return cd(Lsym[2 * t], Lsym[2 * t + 1]);
  };
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s)
          if (std::abs(S(p, q, r, s) - std::conj(S(r, s, p, q))) > 1e-12 * std::max(1.0, lmax))
            return fail(QB_EINVAL, "the symmetrised coupling is not Hermitian: L_{pq;rs} != conj(L_{rs;pq})");
  return QB_OK;
}

// Builds the fill counts, ranking table, coupling combinations and the
// shared-memory image of the space.
static int build_tables(Space& sp) {
  const int M = sp.M, nmax = sp.nmax, Q = sp.Q;
  // cnt[m][n][k]: fillings of modes m..M-1 with n particles, sum_i i n_i = k mod Q.
  // With Q = (M-1) nmax + 1 no momentum sum of the space wraps: the counts, the
  // ranking table and the coupling combinations below are those of exact
  // conservation, and a wrapped (negative) index lands on a zero count.
  auto CI = [&](int m, int n, int k) { return ((size_t)m * (nmax + 1) + n) * Q + k; };
  sp.cnt.assign((size_t)(M + 1) * (nmax + 1) * Q, 0);
  sp.cnt[CI(M, 0, 0)] = 1;
  for (int m = M - 1; m >= 0; --m)
    for (int n = 0; n <= nmax; ++n)
      for (int k = 0; k < Q; ++k) {
        uint64_t acc = 0;
        for (int v = 0; v <= n; ++v) {
          acc += sp.cnt[CI(m + 1, n - v, modp((long long)k - (long long)m * v, Q))];
          if (acc >= (1ull << 62)) acc = (1ull << 62);
        }
        sp.cnt[CI(m, n, k)] = acc;
      }
  for (uint64_t v : sp.cnt)
    if (v >= (1ull << 31)) return fail(QB_EUNSUPPORTED, "a sub-sector count reaches 2^31; reduce n_max");

  Tables& t = sp.t;
  t.M = M;
  t.Q = Q;
  t.exact = sp.exact;
  t.nmax = nmax;
  t.rem_w = nmax + 5;
  t.n_ann = M * (M + 1) / 2;
  const int twoQ = 2 * Q;

  // annihilation pairs (r <= s) and their creation partners (p <= q) in the same
  // momentum class, excluding the pair itself (those are diagonal)
  auto LS = [&](int p, int q, int r, int s) {
    size_t ix = (((size_t)p * M + q) * M + r) * M + s;
    return cd(sp.Lsym[2 * ix], sp.Lsym[2 * ix + 1]);
  };
  std::vector<int> annR, annS, annStart;
  std::vector<uint32_t> pq;
  std::vector<double> G;
  std::vector<std::vector<int>> delta;  // [combo][16]
  std::vector<std::vector<int>> dex;    // [combo][16] shifts of the compact exact index
  // exact momentum: width of mode m's window of suffix momenta, (M-1-m) nmax + 1
  int exw[16] = {0};
  for (int m = 1; m < M; ++m) exw[m] = (M - 1 - m) * nmax + 1;
  std::vector<double> gd;
  unsigned char pairidx[16][16];
  memset(pairidx, 0xff, sizeof(pairidx));
  bool cplx = false;
  for (int r = 0; r < M; ++r)
    for (int s = r; s < M; ++s) {
      int a = (int)annR.size();
      pairidx[r][s] = pairidx[s][r] = (unsigned char)a;
      annR.push_back(r);
      annS.push_back(s);
      annStart.push_back((int)pq.size());
      double mrs = (r == s) ? 1.0 : 2.0;
      gd.push_back(mrs * mrs * LS(r, s, r, s).real());
      int k = (r + s) % Q;
      for (int p = 0; p < M; ++p)
        for (int q = p; q < M; ++q) {
          if ((p + q) % Q != k || (p == r && q == s)) continue;
          double mpq = (p == q) ? 1.0 : 2.0;
          // combos with a zero coupling are kept: for odd M every pair then has
          // (M-1)/2 partners, which the specialised stage kernels unroll
          cd g = std::conj(mpq * mrs * LS(p, q, r, s));
          if (g.imag() != 0.0) cplx = true;
          int lo = std::min(r, p), hi = std::max(s, q);
          pq.push_back((uint32_t)p | ((uint32_t)q << 8) | ((uint32_t)lo << 16) | ((uint32_t)hi << 24));
          G.push_back(g.real());
          G.push_back(g.imag());
          std::vector<int> d(16, 0);
          int dn[16] = {0};
          dn[r] -= 1;
          dn[s] -= 1;
          dn[p] += 1;
          dn[q] += 1;
          std::vector<int> dx(16, 0);
          for (int m = lo + 1; m <= hi; ++m) {
            int dc = 0, dk = 0;
            for (int e = m; e < M; ++e) {
              dc += dn[e];
              dk += dn[e] * e;
            }
            d[m] = dc * twoQ + modp(dk, Q);
            // compact exact index: row (rem) by dc, column (skr - m rem) by dk - m dc
            dx[m] = dc * exw[m] + dk - m * dc;
          }
          delta.push_back(d);
          dex.push_back(dx);
        }
    }
  annStart.push_back((int)pq.size());
  t.n_combo = (int)pq.size();
  t.is_complex = cplx ? 1 : 0;

  // shared-memory image: the stage kernels' tables first after the ranking table
  // (ann .. dsw), so that they stage [E, delta) (mod M) or [ann, sqrt) (exact)
  size_t off = 0;
  t.ncp = (std::max(1, t.n_combo) + 3) & ~3;
  const int nsw = std::max(1, M / 2);  // shift words of a term (modes 1 .. M-1, two per word)
  t.o_cnt = (int)off;
  off = align16(off + sizeof(uint32_t) * (size_t)(M + 1) * (nmax + 1) * Q);
  t.o_E = (int)off;
  off = align16(off + sizeof(int32_t) * (size_t)M * t.rem_w * twoQ);
  // exact momentum: the compact ranking table, where it and the stage kernels' other
  // tables and 12 warps' tiles fit a CTA's shared memory and its shifts fit 16 bits
  t.o_Ex = (int)off;
  t.ex_smem = 0;
  if (sp.exact) {
    size_t exb = 0;
    int dmax = 0;
    for (int m = 1; m < M; ++m) {
      t.ex_w[m] = exw[m];
      t.ex_base[m] = (int)exb;
      exb += sizeof(int32_t) * (size_t)t.rem_w * exw[m];
      dmax = std::max(dmax, 2 * exw[m] + 2 * (M - 1) + 2 * m);
    }
    const size_t rows = 64, iw = (size_t)M;
    size_t wb = iw * rows * 4 + (((size_t)M * rows + 15) & ~(size_t)15) + rows * 4 + rows * 8 + rows +
                2 * (size_t)(t.n_ann + 2) * 4;
    wb = (wb + 15) & ~(size_t)15;
    const size_t rest = 4096 + 32 * (size_t)std::max(1, t.n_combo) * 3 + 16 * (size_t)t.ncp + 1024;
    if (exb + 12 * wb + rest <= 200 * 1024 && dmax <= 32767) {
      t.ex_smem = 1;
      off = align16(off + exb);
    }
  }
  t.o_ann = (int)off;
  off = align16(off + sizeof(int32_t) * (size_t)(t.n_ann + 1));
  t.o_hs = (int)off;
  off = align16(off + sizeof(int32_t) * (size_t)t.n_ann);
  t.o_pairidx = (int)off;
  off = align16(off + 256);
  t.o_Gf = (int)off;
  off = align16(off + sizeof(float) * 4 * (size_t)t.ncp);
  t.o_dsw = (int)off;
  off = align16(off + sizeof(uint32_t) * (size_t)std::max(2, nsw) * t.ncp);
  t.o_dex = (int)off;
  off = align16(off + (t.ex_smem ? (size_t)32 * std::max(1, t.n_combo) : 0));
  t.o_delta = (int)off;
  off = align16(off + (size_t)(sp.exact ? 32 : 16) * std::max(1, t.n_combo));
  t.o_sqrt = (int)off;
  off = align16(off + sizeof(double) * (size_t)(nmax + 3));
  t.o_pq = (int)off;
  off = align16(off + sizeof(uint32_t) * (size_t)std::max(1, t.n_combo));
  t.o_G = (int)off;
  off = align16(off + sizeof(double) * 2 * (size_t)std::max(1, t.n_combo));
  t.o_w = (int)off;
  off = align16(off + sizeof(double) * (size_t)M);
  t.o_gd = (int)off;
  off = align16(off + sizeof(double) * (size_t)t.n_ann);
  t.o_sqf = (int)off;
  off = align16(off + sizeof(float) * 2 * (size_t)(nmax + 3));
  t.blob_bytes = (int)off;
  // mod M: the stage kernels hold two ranking-table byte offsets per 32-bit word, so
  // the table must span at most 64 KB (every space within the other limits does but
  // M = 9 with 97 <= n_max <= 108, whose sectors exceed 2^31 kets anyway)
  t.sw_ok = (!sp.exact && (int64_t)M * t.rem_w * twoQ * 4 <= 65536) ? 1 : 0;
  if (!sp.exact && !t.sw_ok) return fail(QB_EUNSUPPORTED, "the ranking table exceeds 64 KB (reduce n_max)");
  // exact momentum: the fill counts and the ranking table grow with (M-1) n_max
  // and stay in global memory for every kernel
  t.sm_from = sp.exact ? t.o_ann : 0;
  sp.blob.assign(off, 0);
  unsigned char* b = sp.blob.data();
  uint32_t* cnt32 = (uint32_t*)(b + t.o_cnt);
  for (size_t i = 0; i < sp.cnt.size(); ++i) cnt32[i] = (uint32_t)sp.cnt[i];
  int32_t* E = (int32_t*)(b + t.o_E);
  for (int m = 0; m < M; ++m)
    for (int rr = 0; rr < t.rem_w; ++rr)
      for (int kk = 0; kk < twoQ; ++kk) {
        int rem = rr - 2;
        int32_t v = 0;
        if (m >= 1 && rem >= 1 && rem - 1 <= nmax) v = (int32_t)sp.cnt[CI(m - 1, rem - 1, modp(kk - (m - 1), Q))];
        E[((size_t)m * t.rem_w + rr) * twoQ + kk] = v;
      }
  if (t.ex_smem) {
    int32_t* Ex = (int32_t*)(b + t.o_Ex);
    for (int m = 1; m < M; ++m)
      for (int rr = 0; rr < t.rem_w; ++rr)
        for (int c = 0; c < t.ex_w[m]; ++c) {
          const int rem = rr - 2, skr = c + m * rem;
          int32_t v = 0;
          if (rem >= 1 && rem - 1 <= nmax) v = (int32_t)sp.cnt[CI(m - 1, rem - 1, modp(skr - (m - 1), Q))];
          Ex[t.ex_base[m] / 4 + (size_t)rr * t.ex_w[m] + c] = v;
        }
    int16_t* dx = (int16_t*)(b + t.o_dex);
    for (int j = 0; j < t.n_combo; ++j)
      for (int m = 0; m < 16; ++m) dx[(size_t)j * 16 + m] = (int16_t)dex[j][m];
  }
  double* sq = (double*)(b + t.o_sqrt);
  for (int k = 0; k < nmax + 3; ++k) sq[k] = std::sqrt((double)k);
  memcpy(b + t.o_pq, pq.data(), sizeof(uint32_t) * pq.size());
  memcpy(b + t.o_G, G.data(), sizeof(double) * G.size());
  if (sp.exact) {  // int16 shifts (|shift| <= 5Q)
    if (5LL * Q > 32767) return fail(QB_EUNSUPPORTED, "exact momentum: (M-1) n_max too large for 16-bit shifts");
    int16_t* dl = (int16_t*)(b + t.o_delta);
    for (int j = 0; j < t.n_combo; ++j)
      for (int m = 0; m < 16; ++m) dl[(size_t)j * 16 + m] = (int16_t)delta[j][m];
  } else {
    uint8_t* dl = (uint8_t*)(b + t.o_delta);
    for (int j = 0; j < t.n_combo; ++j)
      for (int m = 0; m < 16; ++m) dl[(size_t)j * 16 + m] = (uint8_t)(delta[j][m] + kDeltaBias);
  }
  {  // packed byte shifts: a signed sum, so that the low half's borrow is part of the value
    int32_t* dw = (int32_t*)(b + t.o_dsw);
    for (int j = 0; j < t.n_combo; ++j)
      for (int k = 0; k < std::max(2, nsw); ++k) {
        const int lo = delta[j][2 * k + 1], hi = (2 * k + 2 < 16) ? delta[j][2 * k + 2] : 0;
        const int32_t v = (int32_t)(4 * lo + 65536 * 4 * hi);
        if (k < 2)
          dw[2 * (size_t)j + k] = v;  // words 0, 1 side by side
        else
          dw[(size_t)k * t.ncp + j] = v;  // word k >= 2: column k - 2 after the ncp pairs
      }
  }
  memcpy(b + t.o_ann, annStart.data(), sizeof(int32_t) * annStart.size());
  {  // first combo of each pair whose creation pair comes after it (partners ascend)
    int32_t* hs = (int32_t*)(b + t.o_hs);
    for (int a = 0; a < t.n_ann; ++a) {
      int j = annStart[a];
      while (j < annStart[a + 1] && (int)pairidx[pq[j] & 0xff][(pq[j] >> 8) & 0xff] < a) ++j;
      hs[a] = j;
    }
  }
  memcpy(b + t.o_pairidx, pairidx, 256);
  memcpy(b + t.o_w, sp.w.data(), sizeof(double) * M);
  memcpy(b + t.o_gd, gd.data(), sizeof(double) * gd.size());
  // double-float copies: x = hi + lo with hi = fl32(x), lo = fl32(x - hi)
  auto split = [](double x, float* out) {
    float h = (float)x;
    out[0] = h;
    out[1] = (float)(x - (double)h);
  };
  float* sqf = (float*)(b + t.o_sqf);
  for (int k = 0; k < nmax + 3; ++k) split(std::sqrt((double)k), sqf + 2 * k);
  float* Gf = (float*)(b + t.o_Gf);
  for (int j = 0; j < t.n_combo; ++j) {
    split(G[2 * j], Gf + 2 * j);
    split(G[2 * j + 1], Gf + 2 * ((size_t)t.ncp + j));
  }
  return QB_OK;
}

// rank of an occupation vector within the space (host mirror of the device
// ranking, used for number-state initialisation); -1 if absent
static int64_t host_rank(const Space& sp, const int* occ) {
  const int M = sp.M;
  int N = 0;
  long long K = 0;
  for (int i = 0; i < M; ++i) {
    if (occ[i] < 0) return -1;
    N += occ[i];
    K += (long long)i * occ[i];
  }
  if (N > sp.nmax || N < 0) return -1;
  const int Q = sp.Q;
  int Kk = modp(K, Q);
  int sid = sp.secOf[(size_t)N * Q + Kk];
  if (sid < 0) return -1;
  auto CI = [&](int m, int n, int k) { return ((size_t)m * (sp.nmax + 1) + n) * Q + k; };
  int64_t sum = 0;
  int rem = 0;
  long long kr = 0;
  for (int m = M - 1; m >= 1; --m) {
    rem += occ[m];
    kr += (long long)m * occ[m];
    if (rem >= 1) sum += (int64_t)sp.cnt[CI(m - 1, rem - 1, modp(kr - (m - 1), Q))];
  }
  return sp.secOff[sid] + sp.secDim[sid] - 1 - sum;
}

// ---------------------------------------------------------------- eigensolve

// Eigen-decomposition of a Hermitian n x n matrix (n <= QB_MAX_MODES) by cyclic
// Jacobi rotations on its real 2n x 2n symmetric embedding [[Re, -Im], [Im, Re]].
// Every eigenvalue appears twice there; eig receives the n distinct-slot values
// ascending, vec the unit eigenvector of the largest one.
static void hermitian_eig(int n, const double* A /*[n*n] complex*/, double* eig, double* vec /*[n] complex*/) {
  const int m = 2 * n;
  std::vector<double> S((size_t)m * m), V((size_t)m * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double re = A[2 * (i * n + j)], im = A[2 * (i * n + j) + 1];
      S[(size_t)i * m + j] = re;
      S[(size_t)(i + n) * m + (j + n)] = re;
      S[(size_t)(i + n) * m + j] = im;
      S[(size_t)i * m + (j + n)] = -im;
    }
  // symmetrise against rounding in the input
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      double v = 0.5 * (S[(size_t)i * m + j] + S[(size_t)j * m + i]);
      S[(size_t)i * m + j] = S[(size_t)j * m + i] = v;
    }
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double v = S[(size_t)i * m + j] * S[(size_t)i * m + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = S[(size_t)p * m + q];
        if (apq == 0.0) continue;
        double app = S[(size_t)p * m + p], aqq = S[(size_t)q * m + q];
        double theta = (aqq - app) / (2.0 * apq);
        double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          double skp = S[(size_t)k * m + p], skq = S[(size_t)k * m + q];
          S[(size_t)k * m + p] = c * skp - s * skq;
          S[(size_t)k * m + q] = s * skp + c * skq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          double spk = S[(size_t)p * m + k], sqk = S[(size_t)q * m + k];
          S[(size_t)p * m + k] = c * spk - s * sqk;
          S[(size_t)q * m + k] = s * spk + c * sqk;
        }
        for (int k = 0; k < m; ++k) {
          double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return S[(size_t)a * m + a] < S[(size_t)b * m + b]; });
  for (int k = 0; k < n; ++k)
    eig[k] = 0.5 * (S[(size_t)order[2 * k] * m + order[2 * k]] + S[(size_t)order[2 * k + 1] * m + order[2 * k + 1]]);
  int top = order[m - 1];
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    double x = V[(size_t)i * m + top], y = V[(size_t)(i + n) * m + top];
    vec[2 * i] = x;
    vec[2 * i + 1] = y;
    nrm += x * x + y * y;
  }
  nrm = std::sqrt(nrm);
  for (int i = 0; i < 2 * n; ++i) vec[i] /= nrm;
}

// Derived observables of Sec. II C-E from the raw moments.
void derive(int M, const double* raw, qb_obs* o) {
  memset(o, 0, sizeof(*o));
  double nrm = raw[0];
  o->norm = nrm;
  o->N = raw[1] / nrm;
  o->H = raw[2] / nrm;
  const double* A = raw + 4;
  const double* Mm = A + 2 * M;
  const double* AA = Mm + 2 * M * M;
  std::vector<cd> a(M), Mij((size_t)M * M), aa((size_t)M * M);
  for (int i = 0; i < M; ++i) a[i] = cd(A[2 * i], A[2 * i + 1]) / nrm;
  for (int i = 0; i < M * M; ++i) Mij[i] = cd(Mm[2 * i], Mm[2 * i + 1]) / nrm;
  // <a_k a_l> is symmetric; the device fills k <= l only
  for (int k = 0; k < M; ++k)
    for (int l = 0; l < M; ++l) {
      const int u = (k <= l) ? k * M + l : l * M + k;
      aa[(size_t)k * M + l] = cd(AA[2 * u], AA[2 * u + 1]) / nrm;
    }
  for (int i = 0; i < M; ++i) {
    o->a[2 * i] = a[i].real();
    o->a[2 * i + 1] = a[i].imag();
  }
  std::vector<double> mflat(2 * (size_t)M * M);
  for (int i = 0; i < M * M; ++i) {
    o->Mij[2 * i] = mflat[2 * i] = Mij[i].real();
    o->Mij[2 * i + 1] = mflat[2 * i + 1] = Mij[i].imag();
    o->aa[2 * i] = aa[i].real();
    o->aa[2 * i + 1] = aa[i].imag();
  }
  double ntot = 0.0, dsum = 0.0;
  for (int j = 0; j < M; ++j) {
    ntot += Mij[(size_t)j * M + j].real();
    dsum += Mij[(size_t)j * M + j].real() - std::norm(a[j]);
  }
  o->n_tot = ntot;
  o->Q = dsum / ntot;
  hermitian_eig(M, mflat.data(), o->eig, o->xi);
  o->lam_p = o->eig[M - 1];
  o->PO = 1.0 - o->lam_p / ntot;
  o->gap = (M > 1) ? o->eig[M - 1] - o->eig[M - 2] : INFINITY;
  for (int i = 0; i < M; ++i) {
    double d = Mij[(size_t)i * M + i].real() - std::norm(a[i]);
    cd var = aa[(size_t)i * M + i] - a[i] * a[i];
    o->Vminus[i] = 1.0 + 2.0 * d - 2.0 * std::abs(var);
  }
  std::vector<cd> xi(M);
  for (int k = 0; k < M; ++k) xi[k] = cd(o->xi[2 * k], o->xi[2 * k + 1]);
  cd dd = 0, var = 0;
  for (int k = 0; k < M; ++k)
    for (int l = 0; l < M; ++l) {
      dd += std::conj(xi[k]) * xi[l] * (Mij[(size_t)k * M + l] - std::conj(a[k]) * a[l]);
      var += xi[k] * xi[l] * (aa[(size_t)k * M + l] - a[k] * a[l]);
    }
  o->Vminus_p = 1.0 + 2.0 * dd.real() - 2.0 * std::abs(var);
}

double log2_max_ket_weight(int M, int N) {
  // N! / prod n_m! is largest for the most even occupation: N mod M modes hold
  // floor(N / M) + 1 particles, the rest floor(N / M)
  const int q = N / M, r = N % M;
  const double ln = std::lgamma(N + 1.0) - r * std::lgamma(q + 2.0) - (M - r) * std::lgamma(q + 1.0);
  return 0.5 * ln / std::log(2.0);
}

}  // namespace qb

using namespace qb;

extern "C" {

const char* qb_last_error(void) { return g_err.c_str(); }

int qb_sector_build(const qb_model* model, int n_min, int n_max, const int* p_list, int n_p, qb_space** out) {
  if (!out) return fail(QB_EINVAL, "out must be non-NULL");
  *out = nullptr;
  Space* sp = new (std::nothrow) Space();
  if (!sp) return fail(QB_ENOMEM, "host allocation failed");
  int rc = prepare_model(model, sp->w, sp->Lsym);
  if (rc) {
    delete sp;
    return rc;
  }
  const int M = model->M;
  sp->M = M;
  if (n_min < 0 || n_max < n_min) {
    delete sp;
    return fail(QB_EINVAL, "need 0 <= n_min <= n_max");
  }
  int bits = 1;
  while ((1 << bits) <= n_max) ++bits;
  if (M * bits > 64 || n_max > 250) {
    delete sp;
    return fail(QB_EUNSUPPORTED, "occupation vectors do not pack into 64 bits (M * bits(n_max) > 64)");
  }
  // the stages hold psi / w(n) as fp32 pairs; the centred weights of the deepest sector
  // must stay within the range that keeps them exact (log2 w_max(n_max) <= 160)
  if (log2_max_ket_weight(M, n_max) > kMaxLog2KetWeight) {
    delete sp;
    return fail(QB_EUNSUPPORTED, "ket weights sqrt(N!/prod n!) of the deepest sector exceed 2^160 (reduce n_max): "
                                 "the weighted stage vectors would leave the fp32 exponent range");
  }
  sp->nmin = n_min;
  sp->nmax = n_max;
  sp->exact = model->exact_momentum ? 1 : 0;
  // exact: a modulus above every momentum sum (and above 2(M-1), so that pair
  // momenta never wrap either)
  sp->Q = sp->exact ? std::max((M - 1) * n_max + 1, 2 * M - 1) : M;
  rc = build_tables(*sp);
  if (rc) {
    delete sp;
    return rc;
  }
  std::vector<int> Ps;
  if (p_list) {
    if (n_p < 0) {
      delete sp;
      return fail(QB_EINVAL, "n_p must be >= 0");
    }
    for (int i = 0; i < n_p; ++i) Ps.push_back(sp->exact ? p_list[i] : modp(p_list[i], M));
    std::sort(Ps.begin(), Ps.end());
    Ps.erase(std::unique(Ps.begin(), Ps.end()), Ps.end());
  } else if (sp->exact) {
    // every label sum reachable with N <= n_max: sum_i (i - c) n_i in [-c n_max, (M-1-c) n_max]
    const int c0 = label_shift(M);
    for (int P = -c0 * n_max; P <= (M - 1 - c0) * n_max; ++P) Ps.push_back(P);
  } else {
    for (int P = 0; P < M; ++P) Ps.push_back(P);
  }
  const int c = label_shift(M);
  const int Q = sp->Q;
  sp->secOf.assign((size_t)(n_max + 1) * Q, -1);
  sp->secOff.push_back(0);
  for (int N = n_min; N <= n_max; ++N)
    for (int P : Ps) {
      // index momentum K = sum_i i n_i = P + c N; exact: must lie in [0, (M-1) N]
      const long long Kx = (long long)P + (long long)c * N;
      if (sp->exact && (Kx < 0 || Kx > (long long)(M - 1) * N)) continue;
      int K = modp(Kx, Q);
      uint64_t D = sp->cnt[((size_t)0 * (n_max + 1) + N) * Q + K];
      if (D == 0) continue;
      sp->secOf[(size_t)N * Q + K] = (int)sp->secN.size();
      sp->secN.push_back(N);
      sp->secP.push_back(P);
      sp->secK.push_back(K);
      sp->secDim.push_back((int64_t)D);
      sp->secOff.push_back(sp->secOff.back() + (int64_t)D);
      sp->maxDim = std::max(sp->maxDim, (int64_t)D);
    }
  if (sp->secN.empty()) {
    delete sp;
    return fail(QB_EINVAL, "no non-empty sector in the requested range");
  }
  rc = device_setup(*sp);
  if (rc) {
    qb_space_free(reinterpret_cast<qb_space*>(sp));
    return rc;
  }
  *out = reinterpret_cast<qb_space*>(sp);
  return QB_OK;
}

void qb_space_free(qb_space* space) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return;
  cudaFree(sp->d_blob);
  cudaFree(sp->d_secOff);
  cudaFree(sp->d_secN);
  cudaFree(sp->d_secK);
  cudaFree(sp->d_secOf);
  cudaFree(sp->d_scratch);
  cudaFree(sp->d_diag);
  cudaFree(sp->d_obsf);
  cudaFree(sp->d_wtab);
  cudaFree(sp->d_occ);
  cudaFree(sp->d_wi);
  if (sp->capture_stream) cudaStreamDestroy(sp->capture_stream);
  if (sp->side_stream) cudaStreamDestroy(sp->side_stream);
  if (sp->ev_fork) cudaEventDestroy(sp->ev_fork);
  if (sp->ev_join) cudaEventDestroy(sp->ev_join);
  delete sp;
}

int qb_space_info(const qb_space* space, int64_t* total_states, int* n_sectors, int64_t* max_dim) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (total_states) *total_states = sp->secOff.back();
  if (n_sectors) *n_sectors = (int)sp->secN.size();
  if (max_dim) *max_dim = sp->maxDim;
  return QB_OK;
}

int qb_space_sectors(const qb_space* space, int* N, int* P, int64_t* dim, int64_t* offset) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  for (size_t i = 0; i < sp->secN.size(); ++i) {
    if (N) N[i] = sp->secN[i];
    if (P) P[i] = sp->secP[i];
    if (dim) dim[i] = sp->secDim[i];
    if (offset) offset[i] = sp->secOff[i];
  }
  return QB_OK;
}

int qb_space_basis(const qb_space* space, int64_t first, int64_t count, int* d_occ, void* stream) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (first < 0 || count < 0 || first + count > sp->secOff.back())
    return fail(QB_EINVAL, "ket range outside the space");
  if (count == 0) return QB_OK;
  if (!d_occ) return fail(QB_EINVAL, "d_occ is NULL");
  return launch_unrank(*sp, first, count, d_occ, stream);
}

int qb_space_rank(const qb_space* space, const int* d_occ, int64_t count, int64_t* d_index, void* stream) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (count < 0) return fail(QB_EINVAL, "count < 0");
  if (count == 0) return QB_OK;
  if (!d_occ || !d_index) return fail(QB_EINVAL, "NULL device pointer");
  return launch_rank(*sp, d_occ, count, d_index, stream);
}

int qb_space_terms(const qb_space* space, int64_t* terms, int64_t* tuples, void* stream) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp || !terms) return fail(QB_EINVAL, "space and terms must be non-NULL");
  return launch_terms(*sp, terms, tuples, stream);
}

static int check_state_ptr(const void* p) {
  if (!p) return fail(QB_EINVAL, "state pointer is NULL");
  if (((uintptr_t)p) & 15) return fail(QB_EINVAL, "state pointer must be 16-byte aligned");
  return QB_OK;
}

int qb_init_number(qb_space* space, const int* occ, void* d_psi, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !occ) return fail(QB_EINVAL, "space and occ must be non-NULL");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  int64_t k = host_rank(*sp, occ);
  if (k < 0) return fail(QB_EINVAL, "the occupation vector is not a ket of the space");
  return launch_number(*sp, k, d_psi, stream);
}

// table[i][v] = prefactor_i * zeta_i^v / sqrt(v!) for v = 0..nmax, as complex
static void amp_table(const Space& sp, const double* z, double scale, double mode_pref_log, std::vector<double>& tab,
                      bool coherent) {
  const int M = sp.M, V = sp.nmax + 1;
  tab.assign(2 * (size_t)M * V, 0.0);
  for (int i = 0; i < M; ++i) {
    cd zi = cd(z[2 * i], z[2 * i + 1]) * scale;
    double r = std::abs(zi), th = std::arg(zi);
    double pref = coherent ? -0.5 * r * r : 0.0;
    for (int v = 0; v < V; ++v) {
      double re = 0.0, im = 0.0;
      if (v == 0) {
        re = std::exp(pref);
      } else if (r > 0.0) {
        double lg = pref + v * std::log(r) - 0.5 * std::lgamma((double)v + 1.0);
        double mag = std::exp(lg);
        re = mag * std::cos(v * th);
        im = mag * std::sin(v * th);
      }
      tab[2 * ((size_t)i * V + v)] = re;
      tab[2 * ((size_t)i * V + v) + 1] = im;
    }
  }
  (void)mode_pref_log;
}

int qb_init_coherent(qb_space* space, const double* z, void* d_psi, double* kept_norm, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !z) return fail(QB_EINVAL, "space and z must be non-NULL");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  for (int i = 0; i < 2 * sp->M; ++i)
    if (!std::isfinite(z[i])) return fail(QB_EINVAL, "z has a non-finite entry");
  std::vector<double> tab;
  amp_table(*sp, z, 1.0, 0.0, tab, true);
  double n2 = 0.0;
  rc = launch_init_table(*sp, tab.data(), -1, d_psi, &n2, stream);
  if (rc) return rc;
  if (!(n2 > 0.0)) return fail(QB_EINVAL, "the coherent state has no weight on the space");
  if (kept_norm) *kept_norm = n2;
  return launch_scale(*sp, d_psi, 1.0 / std::sqrt(n2), stream);
}

int qb_init_field_number(qb_space* space, const double* z, int n_tot, void* d_psi, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !z) return fail(QB_EINVAL, "space and z must be non-NULL");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  double zz = 0.0;
  for (int i = 0; i < sp->M; ++i) {
    if (!std::isfinite(z[2 * i]) || !std::isfinite(z[2 * i + 1])) return fail(QB_EINVAL, "z has a non-finite entry");
    zz += z[2 * i] * z[2 * i] + z[2 * i + 1] * z[2 * i + 1];
  }
  if (!(zz > 0.0)) return fail(QB_EINVAL, "z must be nonzero");
  if (n_tot < sp->nmin || n_tot > sp->nmax) return fail(QB_EINVAL, "n_tot is outside the space");
  std::vector<double> tab;
  amp_table(*sp, z, 1.0 / std::sqrt(zz), 0.0, tab, false);
  // sqrt(n_tot!) folded into mode 0's table
  double pref = std::exp(0.5 * std::lgamma((double)n_tot + 1.0));
  for (int v = 0; v <= sp->nmax; ++v) {
    tab[2 * v] *= pref;
    tab[2 * v + 1] *= pref;
  }
  double n2 = 0.0;
  rc = launch_init_table(*sp, tab.data(), n_tot, d_psi, &n2, stream);
  if (rc) return rc;
  if (!(n2 > 0.0)) return fail(QB_EINVAL, "the field number state has no weight on the space");
  // exact normalisation is 1 by the multinomial theorem on the full sector set;
  // renormalise anyway so that a partial P list still yields a unit vector
  return launch_scale(*sp, d_psi, 1.0 / std::sqrt(n2), stream);
}

int64_t qb_workspace_bytes(const qb_space* space, int batch) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp || batch < 1) return -1;
  return workspace_bytes(*sp, batch);
}

int qb_hpsi(qb_space* space, const void* d_psi, void* d_out, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  rc = check_state_ptr(d_out);
  if (rc) return rc;
  if (d_psi == d_out) return fail(QB_EINVAL, "d_psi and d_out must differ");
  return launch_hpsi(*sp, d_psi, d_out, stream);
}

int qb_evolve(qb_space* space, void* d_psi, double dt, int64_t steps, void* d_work, void* stream) {
  double one = 1.0;
  return qb_evolve_batch(space, d_psi, 1, &one, dt, steps, d_work, stream);
}

int qb_evolve_batch(qb_space* space, void* d_psi, int batch, const double* scale, double dt, int64_t steps,
                    void* d_work, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !scale) return fail(QB_EINVAL, "space and scale must be non-NULL");
  if (batch < 1 || batch > 8) return fail(QB_EINVAL, "batch must be in [1, 8]");
  if (steps < 0) return fail(QB_EINVAL, "steps < 0");
  if (!std::isfinite(dt)) return fail(QB_EINVAL, "dt is not finite");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  if (steps == 0) return QB_OK;
  rc = check_state_ptr(d_work);
  if (rc) return rc;
  for (int b = 0; b < batch; ++b)
    if (!std::isfinite(scale[b])) return fail(QB_EINVAL, "scale has a non-finite entry");
  return launch_rk4(*sp, d_psi, batch, scale, dt, steps, d_work, stream);
}

int qb_space_set_resident_max(qb_space* space, int resident_max_kets) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (resident_max_kets < 0) return fail(QB_EINVAL, "resident_max_kets must be >= 0");
  sp->resident_max_kets = resident_max_kets;
  return QB_OK;
}

int qb_space_set_tile_shape(qb_space* space, int shape) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (shape < 0 || shape >= QB_TILE_SHAPES) return fail(QB_EINVAL, "shape must be in [0, QB_TILE_SHAPES)");
  sp->tile_shape = shape;
  return QB_OK;
}

int qb_space_set_order(qb_space* space, int order) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (order < 2 || order > 4) return fail(QB_EINVAL, "order must be 2, 3 or 4");
  sp->order = order;
  return QB_OK;
}

int qb_evolve_plain(qb_space* space, void* d_psi, double dt, int64_t steps, void* d_work, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  if (steps < 0) return fail(QB_EINVAL, "steps < 0");
  if (!std::isfinite(dt)) return fail(QB_EINVAL, "dt is not finite");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  if (steps == 0) return QB_OK;
  rc = check_state_ptr(d_work);
  if (rc) return rc;
  double one = 1.0;
  return launch_rk4(*sp, d_psi, 1, &one, dt, steps, d_work, stream, true);
}

int qb_observables(qb_space* space, const void* d_psi, qb_obs* out, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !out) return fail(QB_EINVAL, "space and out must be non-NULL");
  int rc = check_state_ptr(d_psi);
  if (rc) return rc;
  const int M = sp->M;
  std::vector<double> raw(4 + 2 * M + 4 * (size_t)M * M, 0.0);
  rc = launch_moments(*sp, d_psi, raw.data(), stream);
  if (rc) return rc;
  if (!(raw[0] > 0.0)) return fail(QB_EINVAL, "the state has zero norm");
  derive(M, raw.data(), out);
  return QB_OK;
}

int qb_evolve_observe(qb_space* space, void* d_psi, double dt, int64_t steps, int obs_every, qb_obs* series,
                      void* d_work, void* stream) {
  if (obs_every < 1 || steps < 0 || steps % obs_every != 0)
    return fail(QB_EINVAL, "steps must be a non-negative multiple of obs_every >= 1");
  if (!series) return fail(QB_EINVAL, "series is NULL");
  int64_t nobs = steps / obs_every;
  int rc = qb_observables(space, d_psi, &series[0], stream);
  if (rc) return rc;
  series[0].t = 0.0;
  for (int64_t k = 1; k <= nobs; ++k) {
    rc = qb_evolve(space, d_psi, dt, obs_every, d_work, stream);
    if (rc) return rc;
    rc = qb_observables(space, d_psi, &series[k], stream);
    if (rc) return rc;
    series[k].t = (double)k * obs_every * dt;
  }
  return QB_OK;
}

int qb_breaktime(const double* values, int n, double dt_obs, double thr, double* t_br, int* flag) {
  if (!values || !t_br || !flag || n < 0) return fail(QB_EINVAL, "bad arguments");
  for (int k = 0; k < n; ++k) {
    if (values[k] >= thr) {
      if (k == 0) {
        *t_br = 0.0;
        *flag = QB_AT_START;
      } else {
        double f = (thr - values[k - 1]) / (values[k] - values[k - 1]);
        *t_br = ((double)(k - 1) + f) * dt_obs;
        *flag = QB_CROSSED;
      }
      return QB_OK;
    }
  }
  *t_br = NAN;
  *flag = QB_NOT_CROSSED;
  return QB_OK;
}

int qb_squeezing(const double* vminus, int n, double dt_obs, double thr, double* t_sqz, int* flag, double* v_min,
                 double* t_min) {
  if (!vminus || !t_sqz || !flag || !v_min || !t_min || n < 1 || !(dt_obs > 0.0))
    return fail(QB_EINVAL, "bad arguments");
  *t_sqz = NAN;
  *flag = QB_NOT_CROSSED;
  for (int k = 0; k < n; ++k) {
    if (vminus[k] <= thr) {
      if (k == 0) {
        *t_sqz = 0.0;
        *flag = QB_AT_START;
      } else {
        const double f = (vminus[k - 1] - thr) / (vminus[k - 1] - vminus[k]);
        *t_sqz = ((double)(k - 1) + f) * dt_obs;
        *flag = QB_CROSSED;
      }
      break;
    }
  }
  int kmin = 0;
  for (int k = 1; k < n; ++k)
    if (vminus[k] < vminus[kmin]) kmin = k;
  *v_min = vminus[kmin];
  *t_min = kmin * dt_obs;
  if (kmin > 0 && kmin < n - 1) {
    // vertex of the parabola through (-1, a), (0, b), (1, c) in units of dt_obs
    const double a = vminus[kmin - 1], b = vminus[kmin], c = vminus[kmin + 1];
    const double den = a - 2.0 * b + c;
    if (den > 0.0) {
      const double u = 0.5 * (a - c) / den;  // in [-1/2, 1/2] since b is the smallest
      *t_min = (kmin + u) * dt_obs;
      *v_min = b - 0.25 * (a - c) * u;
    }
  }
  return QB_OK;
}

int qb_interaction_per_occupation(const qb_model* model, const double* z, double* ntot_chi) {
  if (!model || !z || !ntot_chi) return fail(QB_EINVAL, "bad arguments");
  std::vector<double> w, Ls;
  int rc = prepare_model(model, w, Ls);
  if (rc) return rc;
  const int M = model->M;
  std::vector<cd> zz(M);
  double n = 0.0;
  for (int p = 0; p < M; ++p) {
    if (!std::isfinite(z[2 * p]) || !std::isfinite(z[2 * p + 1])) return fail(QB_EINVAL, "z has a non-finite entry");
    zz[p] = cd(z[2 * p], z[2 * p + 1]);
    n += std::norm(zz[p]);
  }
  if (!(n > 0.0)) return fail(QB_EINVAL, "z must be nonzero");
  cd acc = 0.0;
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s) {
          const size_t t = (((size_t)p * M + q) * M + r) * M + s;
          acc += cd(Ls[2 * t], Ls[2 * t + 1]) * std::conj(zz[p]) * std::conj(zz[q]) * zz[r] * zz[s];
        }
  *ntot_chi = acc.real() / n;
  return QB_OK;
}

int qb_fit(const double* x, const double* y, int n, int kind, double* c0, double* c1) {
  if (!x || !y || !c0 || !c1 || n < 2 || (kind != 0 && kind != 1)) return fail(QB_EINVAL, "bad arguments");
  double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
  for (int k = 0; k < n; ++k) {
    if (!(x[k] > 0.0) || (kind == 0 && !(y[k] > 0.0))) return fail(QB_EINVAL, "the fit needs positive data");
    const double u = std::log(x[k]), v = kind == 0 ? std::log(y[k]) : y[k];
    sx += u;
    sy += v;
    sxx += u * u;
    sxy += u * v;
  }
  const double det = n * sxx - sx * sx;
  if (!(det > 0.0)) return fail(QB_EINVAL, "the fit needs two distinct x");
  const double slope = (n * sxy - sx * sy) / det, icpt = (sy - slope * sx) / n;
  *c1 = slope;
  *c0 = kind == 0 ? std::exp(icpt) : icpt;
  return QB_OK;
}

int qb_meanfield(const qb_model* model, const double* z0, double dt, int64_t steps, int every, double* traj) {
  if (!model || !model->w || !model->L || !z0 || !traj || every < 1 || steps < 0)
    return fail(QB_EINVAL, "bad arguments");
  const int M = model->M;
  if (M < 1 || M > QB_MAX_MODES) return fail(QB_EUNSUPPORTED, "M must be in [1, QB_MAX_MODES]");
  std::vector<cd> G((size_t)M * M * M * M);
  for (int k = 0; k < M; ++k)
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r)
        for (int s = 0; s < M; ++s) {
          size_t t1 = (((size_t)k * M + q) * M + r) * M + s, t2 = (((size_t)q * M + k) * M + r) * M + s;
          G[t1] = cd(model->L[2 * t1], model->L[2 * t1 + 1]) + cd(model->L[2 * t2], model->L[2 * t2 + 1]);
        }
  auto rhs = [&](const std::vector<cd>& a, std::vector<cd>& f) {
    for (int k = 0; k < M; ++k) {
      cd acc = model->w[k] * a[k];
      for (int q = 0; q < M; ++q)
        for (int r = 0; r < M; ++r)
          for (int s = 0; s < M; ++s) acc += G[(((size_t)k * M + q) * M + r) * M + s] * std::conj(a[q]) * a[r] * a[s];
      f[k] = cd(0, -1) * acc;
    }
  };
  std::vector<cd> a(M), k1(M), k2(M), k3(M), k4(M), u(M);
  for (int i = 0; i < M; ++i) a[i] = cd(z0[2 * i], z0[2 * i + 1]);
  int64_t row = 0;
  for (int i = 0; i < M; ++i) {
    traj[2 * i] = a[i].real();
    traj[2 * i + 1] = a[i].imag();
  }
  for (int64_t st = 1; st <= steps; ++st) {
    rhs(a, k1);
    for (int i = 0; i < M; ++i) u[i] = a[i] + 0.5 * dt * k1[i];
    rhs(u, k2);
    for (int i = 0; i < M; ++i) u[i] = a[i] + 0.5 * dt * k2[i];
    rhs(u, k3);
    for (int i = 0; i < M; ++i) u[i] = a[i] + dt * k3[i];
    rhs(u, k4);
    for (int i = 0; i < M; ++i) a[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    if (st % every == 0) {
      ++row;
      for (int i = 0; i < M; ++i) {
        traj[2 * (row * M + i)] = a[i].real();
        traj[2 * (row * M + i) + 1] = a[i].imag();
      }
    }
  }
  return QB_OK;
}

}  // extern "C"
