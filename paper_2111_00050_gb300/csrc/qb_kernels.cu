// sm_103a kernels of the qb library: matrix-free sector H psi fused into the
// Horner-form RK4 stages, combinatorial unrank / rank, initial states,
// observable moments with deterministic two-pass reductions.
//
// Paper: Eberhardt, Zamora, Kopp & Abel, arXiv:2111.00050.  The Hamiltonian is
// Eq. (Ham); sectors are the special Hilbert spaces of Sec. III B; the state of
// every sector evolves independently (Sec. III B), so one launch covers all
// sectors of a space (and all members of a batched coupling sweep).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "qb_internal.h"

#include "qb_device.cuh"
#include "qb_stage.cuh"

namespace qb {

// ------------------------------------------------------------ H psi kernels

enum { MODE_HPSI = 0, MODE_STAGE = 1, MODE_DOT = 2 };

struct StageArgs {
  const double2* vin;  // gathered vector(s) [B][total]
  const double2* psi;  // psi(s) [B][total] (stage mode)
  double2* out;        // output(s) [B][total]
  double scale[8];     // two-body scale per member
  double zre;          // stage factor  -i dt / d  = (0, -dt/d): out = psi + (dt/d) * (Im Hv, -Re Hv)
  double* partial;     // MODE_DOT: [gridDim.x][2]
  int* status;         // device status word (bounds violations)
};

template <int MODE, int B, bool CPLX>
__global__ void __launch_bounds__(kBlock) hpsi_kernel(const Tables t, const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x;
  const int M = t.M;
  const int64_t total = t.total;
  double dot_re = 0.0, dot_im = 0.0;

  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    if (g >= total) break;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    const int N = __ldg(t.sec_N + sid), K = __ldg(t.sec_K + sid);
    const int64_t me = setup_row(t, v, rs, N, K, D, g - off);
    if (me != g - off) atomicOr(a.status, 2);

    const uint8_t* occ = rs.occ + tid;
    const int32_t* idx = rs.idx + tid;
    const int32_t* pe = rs.pe + tid;
    uint32_t occmask = 0, twomask = 0;
    double dw = 0.0;
    for (int m = 0; m < M; ++m) {
      int nm = occ[m * kBlock];
      occmask |= (nm >= 1 ? 1u : 0u) << m;
      twomask |= (nm >= 2 ? 1u : 0u) << m;
      dw += v.w[m] * nm;
    }
    const int64_t rank_base = D - 1 - pe[(M - 1) * kBlock];
    double dl = 0.0;
    double acc_re[B], acc_im[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc_re[b] = acc_im[b] = 0.0;

    // flattened iteration over annihilation pairs r <= s with n_r (n_s - [r==s]) > 0
    uint32_t rm = occmask, sm = 0;
    int r = 0;
    while (true) {
      if (sm == 0) {
        if (rm == 0) break;
        r = __ffs(rm) - 1;
        rm &= rm - 1;
        sm = occmask & (~0u << r);
        if (!((twomask >> r) & 1u)) sm &= ~(1u << r);
        if (sm == 0) continue;
      }
      const int s = __ffs(sm) - 1;
      sm &= sm - 1;
      const int ai = v.pairidx[r * 16 + s];
      const int nr = occ[r * kBlock], ns = occ[s * kBlock];
      const double A = v.sq[nr] * v.sq[ns - (r == s ? 1 : 0)];
      dl += v.gd[ai] * (double)(nr * (ns - (r == s ? 1 : 0)));
      double pr[B], pi[B];
#pragma unroll
      for (int b = 0; b < B; ++b) pr[b] = pi[b] = 0.0;
      const int j1 = v.ann[ai + 1];
      for (int j = v.ann[ai]; j < j1; ++j) {
        const uint32_t w4 = v.pq[j];
        const int p = w4 & 0xff, q = (w4 >> 8) & 0xff, lo = (w4 >> 16) & 0xff, hi = w4 >> 24;
        const int np_ = occ[p * kBlock], nq = occ[q * kBlock];
        const double Bf = v.sq[np_ + 1] * v.sq[nq + 1 + (p == q ? 1 : 0)];
        int64_t rk = rank_base + pe[hi * kBlock] - pe[lo * kBlock];
        for (int m = lo + 1; m <= hi; ++m) rk -= v.E[idx[m * kBlock] + delta_shift(t, v, j, m)];
        if (rk < 0 || rk >= D) {
          atomicOr(a.status, 1);
          rk = 0;
        }
        const double cr = v.G[2 * j] * Bf;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const double2 x = __ldg(a.vin + (size_t)b * total + off + rk);
          if (CPLX) {
            const double ci = v.G[2 * j + 1] * Bf;
            pr[b] += cr * x.x - ci * x.y;
            pi[b] += cr * x.y + ci * x.x;
          } else {
            pr[b] += cr * x.x;
            pi[b] += cr * x.y;
          }
        }
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        acc_re[b] += A * pr[b];
        acc_im[b] += A * pi[b];
      }
    }

#pragma unroll
    for (int b = 0; b < B; ++b) {
      const double sc = a.scale[b];
      const double2 x = a.vin[(size_t)b * total + g];
      const double dg = dw + sc * dl;
      const double hr = dg * x.x + sc * acc_re[b];
      const double hi = dg * x.y + sc * acc_im[b];
      if (MODE == MODE_HPSI) {
        a.out[(size_t)b * total + g] = make_double2(hr, hi);
      } else if (MODE == MODE_STAGE) {
        const double2 p0 = a.psi[(size_t)b * total + g];
        // psi + (-i dt/d) * Hv,  zre = dt/d
        a.out[(size_t)b * total + g] = make_double2(p0.x + a.zre * hi, p0.y - a.zre * hr);
      } else {
        // <x | Hx> contribution: conj(x) * Hx
        dot_re += x.x * hr + x.y * hi;
        dot_im += x.x * hi - x.y * hr;
      }
    }
  }

  if (MODE == MODE_DOT) {
    __shared__ double red[2][kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) {
      dot_re += __shfl_down_sync(0xffffffffu, dot_re, o);
      dot_im += __shfl_down_sync(0xffffffffu, dot_im, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = dot_re;
      red[1][tid >> 5] = dot_im;
    }
    __syncthreads();
    if (tid == 0) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < kBlock / 32; ++k) {
        sr += red[0][k];
        si += red[1][k];
      }
      a.partial[2 * blockIdx.x] = sr;
      a.partial[2 * blockIdx.x + 1] = si;
    }
  }
}


// psi (FP64) -> double-float copy
__global__ void to_df_kernel(const double2* psi, float4* out, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = psi[k];
    out[k] = df_pack(df_of(x.x), df_of(x.y));
  }
}

// psi (FP64, [B][total]) -> double-float copy in the weighted basis, f = psi / w(n),
// with the inverse weights of the per-ket table (coalesced, no unranking)
template <int MT>
__global__ void __launch_bounds__(256) to_dfw_kernel(const Tables t, const double2* psi, float4* out, int B) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < t.total; g += (int64_t)gridDim.x * blockDim.x) {
    const double wi = __ldg(t.wi + g);
    for (int b = 0; b < B; ++b) {
      const double2 x = psi[(size_t)b * t.total + g];
      out[(size_t)b * t.total + g] = df_pack(df_of(x.x * wi), df_of(x.y * wi));
    }
  }
}

// per-ket diagonal of H, one-body and two-body parts, as double-float pairs; the
// packed occupations and the inverse ket weight of every ket
__global__ void __launch_bounds__(kBlock) diag_kernel(const Tables t, float4* diag, uint64_t* occ, double* wi) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x, M = t.M;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < t.total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    if (g >= t.total) break;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    setup_row(t, v, rs, __ldg(t.sec_N + sid), __ldg(t.sec_K + sid), D, g - off);
    double dw = 0.0, dl = 0.0;
    uint64_t word = 0;
    for (int r = 0; r < M; ++r) {
      const int nr = rs.occ[r * kBlock + tid];
      word |= (uint64_t)nr << (r * t.occ_bits);
      dw += v.w[r] * nr;
      for (int s2 = r; s2 < M; ++s2) {
        const int ns = rs.occ[s2 * kBlock + tid] - (r == s2 ? 1 : 0);
        if (nr >= 1 && ns >= 1) dl += v.gd[v.pairidx[r * 16 + s2]] * (double)(nr * ns);
      }
    }
    const dfl a = df_of(dw), b = df_of(dl);
    diag[g] = make_float4(a.h, a.l, b.h, b.l);
    occ[g] = word;
    wi[g] = ket_weight<0>(t, rs.occ + tid, kBlock).y;
  }
}

// ------------------------------------------------------------- small kernels

__global__ void __launch_bounds__(kBlock) unrank_kernel(const Tables t, int64_t first, int64_t count, int* occ_out,
                                                         int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < count; base += (int64_t)gridDim.x * kBlock) {
    const int64_t k = base + tid;
    if (k >= count) break;
    const int64_t g = first + k;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    const int64_t me = setup_row(t, v, rs, __ldg(t.sec_N + sid), __ldg(t.sec_K + sid), D, g - off);
    if (me != g - off) atomicOr(status, 2);
    for (int m = 0; m < t.M; ++m) occ_out[k * t.M + m] = rs.occ[m * kBlock + tid];
  }
}

__global__ void __launch_bounds__(kBlock) rank_kernel(const Tables t, const int* occ_in, int64_t count,
                                                       int64_t* index_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const int M = t.M, V = t.nmax + 1;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    int N = 0, K = 0;
    bool ok = true;
    for (int m = 0; m < M; ++m) {
      int nm = occ_in[k * M + m];
      if (nm < 0 || nm > t.nmax) ok = false;
      N += nm;
      K = (K + m * (nm < 0 ? 0 : nm)) % t.Q;
    }
    int64_t res = -1;
    if (ok && N <= t.nmax) {
      int sid = __ldg(t.sec_of + N * t.Q + K);
      if (sid >= 0) {
        const int64_t off = __ldg(t.sec_off + sid), D = __ldg(t.sec_off + sid + 1) - off;
        int64_t sum = 0;
        int rem = 0, kr = 0;
        for (int m = M - 1; m >= 1; --m) {
          int nm = occ_in[k * M + m];
          rem += nm;
          kr = (kr + m * nm) % t.Q;
          if (rem >= 1)
            sum += v.cnt[((size_t)(m - 1) * V + rem - 1) * t.Q + (((kr - (m - 1)) % t.Q) + t.Q) % t.Q];
        }
        res = off + D - 1 - sum;
      }
    }
    index_out[k] = res;
  }
}

__global__ void __launch_bounds__(kBlock) terms_kernel(const Tables t, unsigned long long* out /*[2]*/) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x, M = t.M;
  unsigned long long terms = 0, tuples = 0;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < t.total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    if (g >= t.total) break;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    setup_row(t, v, rs, __ldg(t.sec_N + sid), __ldg(t.sec_K + sid), D, g - off);
    terms += 1;  // diagonal element
    for (int r = 0; r < M; ++r)
      for (int s = r; s < M; ++s) {
        int nr = rs.occ[r * kBlock + tid], ns = rs.occ[s * kBlock + tid];
        if (nr < 1 || ns - (r == s ? 1 : 0) < 1) continue;
        int ai = v.pairidx[r * 16 + s];
        unsigned long long mrs = (r == s) ? 1 : 2;
        if (v.gd[ai] != 0.0) tuples += mrs * mrs;
        for (int j = v.ann[ai]; j < v.ann[ai + 1]; ++j) {
          if (v.G[2 * j] == 0.0 && v.G[2 * j + 1] == 0.0) continue;
          uint32_t w4 = v.pq[j];
          int p = w4 & 0xff, q = (w4 >> 8) & 0xff;
          terms += 1;
          tuples += mrs * ((p == q) ? 1ull : 2ull);
        }
      }
  }
  for (int o = 16; o > 0; o >>= 1) {
    terms += __shfl_down_sync(0xffffffffu, terms, o);
    tuples += __shfl_down_sync(0xffffffffu, tuples, o);
  }
  if ((tid & 31) == 0) {
    atomicAdd(out, terms);
    atomicAdd(out + 1, tuples);
  }
}

// amplitude = prod_i table[i][n_i] (complex), zero outside N == only_N (if >= 0);
// per-block partial sums of |amplitude|^2
__global__ void __launch_bounds__(kBlock) init_table_kernel(const Tables t, const double2* table, int only_N,
                                                             double2* psi, double* partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x, M = t.M, V = t.nmax + 1;
  double n2 = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < t.total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    if (g >= t.total) break;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    const int N = __ldg(t.sec_N + sid);
    double re = 0.0, im = 0.0;
    if (only_N < 0 || N == only_N) {
      setup_row(t, v, rs, N, __ldg(t.sec_K + sid), D, g - off);
      re = 1.0;
      for (int m = 0; m < M; ++m) {
        const double2 f = __ldg(table + (size_t)m * V + rs.occ[m * kBlock + tid]);
        const double nr = re * f.x - im * f.y;
        im = re * f.y + im * f.x;
        re = nr;
      }
    }
    psi[g] = make_double2(re, im);
    n2 += re * re + im * im;
  }
  __shared__ double red[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, o);
  if ((tid & 31) == 0) red[tid >> 5] = n2;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) s += red[k];
    partial[blockIdx.x] = s;
  }
}

// sums partial[0..n)[0..width) over the first index in a fixed order
__global__ void reduce_partials_kernel(const double* partial, int n, int width, double* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < width; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partial[(size_t)k * width + c];
    out[c] = s;
  }
}

__global__ void scale_kernel(double2* psi, int64_t n, double f) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double2 x = psi[k];
    psi[k] = make_double2(x.x * f, x.y * f);
  }
}

__global__ void number_kernel(double2* psi, int64_t n, int64_t index) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    psi[k] = make_double2(k == index ? 1.0 : 0.0, 0.0);
}

// ---------------------------------------------------------------- moments
//
// Raw moments of Sec. II C-E: norm, <N>, <a_i>, <a_i^dag a_j>, <a_i a_j>.  Each
// row (ket n with amplitude x) contributes conj(psi[target]) * c * x for every
// operator that maps n to a held ket.  Contributions are reduced across the warp
// by shuffles into per-warp shared accumulators, then across warps into one
// partial per block, then over blocks in a fixed order: deterministic.

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__global__ void __launch_bounds__(kBlock) moments_kernel(const Tables t, const double2* psi, double* partial,
                                                          int nmom, int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const size_t blob_al = blob_smem(t);
  const RowScratch rs = row_scratch(smem + blob_al);
  double* acc = reinterpret_cast<double*>(smem + blob_al + ((kRowScratchBytes + 15) & ~15));  // [warps][nmom]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, M = t.M;
  for (int k = tid; k < (kBlock / 32) * nmom; k += kBlock) acc[k] = 0.0;
  __syncthreads();
  double* wacc = acc + (size_t)warp * nmom;
  // layout: [0] norm [1] N [2] H (unused here) [3] pad, a: 4.., Mij: 4+2M.., aa: 4+2M+2M^2..
  const int oA = 4, oM = 4 + 2 * M, oAA = 4 + 2 * M + 2 * M * M;

  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < t.total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    const bool live = g < t.total;
    int N = 0, K = 0;
    double xr = 0.0, xi = 0.0;
    if (live) {
      const int sid = find_sector(t, g);
      const int64_t off = __ldg(t.sec_off + sid);
      const int64_t D = __ldg(t.sec_off + sid + 1) - off;
      N = __ldg(t.sec_N + sid);
      K = __ldg(t.sec_K + sid);
      setup_row(t, v, rs, N, K, D, g - off);
      const double2 x = psi[g];
      xr = x.x;
      xi = x.y;
    }
    const double p2 = xr * xr + xi * xi;
    {
      double c0 = warp_sum(p2), c1 = warp_sum(p2 * N);
      if (lane == 0) {
        wacc[0] += c0;
        wacc[1] += c1;
      }
    }
    // contribution conj(y) * c * x for target index tg (or none)
    auto contrib = [&](int slot, bool has, int64_t tg, double c) {
      double cr = 0.0, ci = 0.0;
      if (has && (tg < 0 || tg >= t.total)) {
        atomicOr(status, 1);
        has = false;
      }
      if (has) {
        const double2 y = psi[tg];
        cr = c * (y.x * xr + y.y * xi);
        ci = c * (y.x * xi - y.y * xr);
      }
      if (__any_sync(0xffffffffu, has)) {
        cr = warp_sum(cr);
        ci = warp_sum(ci);
        if (lane == 0) {
          wacc[slot] += cr;
          wacc[slot + 1] += ci;
        }
      }
    };
    const uint8_t* occ = rs.occ + tid;
    // <a_i>
    for (int i = 0; i < M; ++i) {
      bool has = false;
      int64_t tg = 0;
      double c = 0.0;
      if (live && occ[i * kBlock] >= 1 && N >= 1) {
        const int Kt = ((K - i) % t.Q + t.Q) % t.Q;
        const int sid = __ldg(t.sec_of + (N - 1) * t.Q + Kt);
        if (sid >= 0) {
          const int64_t off = __ldg(t.sec_off + sid), D = __ldg(t.sec_off + sid + 1) - off;
          int e[1] = {i}, dn[1] = {-1};
          tg = off + rank_changed(t, v, rs, 1, e, dn, D);
          c = v.sq[occ[i * kBlock]];
          has = true;
        }
      }
      contrib(oA + 2 * i, has, tg, c);
    }
    // <a_i^dag a_j>
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        bool has = false;
        int64_t tg = 0;
        double c = 0.0;
        if (live && occ[j * kBlock] >= 1) {
          if (i == j) {
            tg = g;
            c = (double)occ[i * kBlock];
            has = true;
          } else {
            const int Kt = ((K - j + i) % t.Q + t.Q) % t.Q;
            const int sid = __ldg(t.sec_of + N * t.Q + Kt);
            if (sid >= 0) {
              const int64_t off = __ldg(t.sec_off + sid), D = __ldg(t.sec_off + sid + 1) - off;
              int e[2] = {j, i}, dn[2] = {-1, 1};
              tg = off + rank_changed(t, v, rs, 2, e, dn, D);
              c = v.sq[occ[j * kBlock]] * v.sq[occ[i * kBlock] + 1];
              has = true;
            }
          }
        }
        contrib(oM + 2 * (i * M + j), has, tg, c);
      }
    // <a_i a_j>, i <= j (the matrix is symmetric)
    for (int i = 0; i < M; ++i)
      for (int j = i; j < M; ++j) {
        bool has = false;
        int64_t tg = 0;
        double c = 0.0;
        if (live && N >= 2) {
          const int ni = occ[i * kBlock], nj = occ[j * kBlock];
          const bool ok = (i == j) ? (ni >= 2) : (ni >= 1 && nj >= 1);
          if (ok) {
            const int Kt = ((K - i - j) % t.Q + t.Q) % t.Q;
            const int sid = __ldg(t.sec_of + (N - 2) * t.Q + Kt);
            if (sid >= 0) {
              const int64_t off = __ldg(t.sec_off + sid), D = __ldg(t.sec_off + sid + 1) - off;
              int e[2] = {i, j}, dn[2] = {(i == j) ? -2 : -1, -1};
              tg = off + rank_changed(t, v, rs, (i == j) ? 1 : 2, e, dn, D);
              c = (i == j) ? v.sq[ni] * v.sq[ni - 1] : v.sq[ni] * v.sq[nj];
              has = true;
            }
          }
        }
        contrib(oAA + 2 * (i * M + j), has, tg, c);
      }
  }
  __syncthreads();
  for (int k = tid; k < nmom; k += kBlock) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += acc[(size_t)w * nmom + k];
    partial[(size_t)blockIdx.x * nmom + k] = s;
  }
}


// ------------------------------------------------------------------ host side

static size_t row_smem(const Tables& t) { return blob_smem(t) + kRowScratchBytes; }

// grid of a persistent row kernel, capped by the scratch sizing

int check_status(const Space& s, cudaStream_t st) {
  int h = 0;
  int* d = reinterpret_cast<int*>(s.d_scratch);  // status word lives at the head of the scratch area
  QB_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  if (h) {
    QB_CUDA(cudaMemsetAsync(d, 0, sizeof(int), st));
    QB_CUDA(cudaStreamSynchronize(st));
    return fail(QB_EINTERNAL, "device-side consistency check failed (status " + std::to_string(h) + ")");
  }
  return QB_OK;
}

int device_setup(Space& s) {
  QB_CUDA(cudaGetDevice(&s.device));
  const size_t nsec = s.secN.size();
  QB_CUDA(cudaMalloc(&s.d_blob, s.blob.size()));
  QB_CUDA(cudaMemcpy(s.d_blob, s.blob.data(), s.blob.size(), cudaMemcpyHostToDevice));
  QB_CUDA(cudaMalloc(&s.d_secOff, sizeof(int64_t) * (nsec + 1)));
  QB_CUDA(cudaMemcpy(s.d_secOff, s.secOff.data(), sizeof(int64_t) * (nsec + 1), cudaMemcpyHostToDevice));
  QB_CUDA(cudaMalloc(&s.d_secN, sizeof(int32_t) * nsec));
  QB_CUDA(cudaMemcpy(s.d_secN, s.secN.data(), sizeof(int32_t) * nsec, cudaMemcpyHostToDevice));
  QB_CUDA(cudaMalloc(&s.d_secK, sizeof(int32_t) * nsec));
  QB_CUDA(cudaMemcpy(s.d_secK, s.secK.data(), sizeof(int32_t) * nsec, cudaMemcpyHostToDevice));
  QB_CUDA(cudaMalloc(&s.d_secOf, sizeof(int32_t) * s.secOf.size()));
  QB_CUDA(cudaMemcpy(s.d_secOf, s.secOf.data(), sizeof(int32_t) * s.secOf.size(), cudaMemcpyHostToDevice));
  Tables& t = s.t;
  t.blob = s.d_blob;
  t.n_sectors = (int)nsec;
  t.sec_off = s.d_secOff;
  t.sec_N = s.d_secN;
  t.sec_K = s.d_secK;
  t.sec_of = s.d_secOf;
  t.total = s.secOff.back();
  if (row_smem(t) + (size_t)(kBlock / 32) * nmoments(s.M) * 8 > 227 * 1024)
    return fail(QB_EUNSUPPORTED, "tables too large for shared memory (reduce n_max or M)");
  // scratch: status + partials for the largest persistent grid of any reduction
  int sms = 0;
  QB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
  const int64_t max_grid = (int64_t)sms * 16;
  s.grid_hpsi = (int)max_grid;
  s.scratch_doubles = scratch_doubles_for(s.M, s.nmax, max_grid);
  QB_CUDA(cudaMalloc(&s.d_scratch, sizeof(double) * s.scratch_doubles));
  QB_CUDA(cudaMemset(s.d_scratch, 0, sizeof(double) * s.scratch_doubles));
  QB_CUDA(cudaMalloc(&s.d_diag, sizeof(float4) * (size_t)t.total));
  QB_CUDA(cudaMalloc(&s.d_obsf, sizeof(float4) * (size_t)t.total));
  QB_CUDA(cudaMalloc(&s.d_occ, sizeof(uint64_t) * (size_t)t.total));
  QB_CUDA(cudaMalloc(&s.d_wi, sizeof(double) * (size_t)t.total));
  t.wi = s.d_wi;
  t.occ_bits = 1;
  while ((1 << t.occ_bits) <= s.nmax) ++t.occ_bits;  // M * occ_bits <= 64 (checked by qb_sector_build)
  t.occ = s.d_occ;
  {
    // sqrt(C(rem, k)): the binomial exactly in 128 bits while it fits (rem <= 125:
    // C(125, 62) < 2^122), then one rounding to double, one correctly rounded sqrt
    // and one division; beyond, by the recurrence C(rem, k) = C(rem, k-1) (rem-k+1) / k
    // in long double (at least 64 significant bits: the accumulated relative error
    // of at most 2 rem roundings stays far below a double's half-ulp)
    const int V = s.nmax + 1;
    std::vector<double2> wt((size_t)V * V, make_double2(0.0, 0.0));
    for (int rem = 0; rem < V; ++rem) {
      unsigned __int128 c = 1;
      long double cl = 1.0L;
      for (int k = 0; k <= rem; ++k) {
        if (k > 0) {
          if (rem <= 125)
            c = c * (unsigned __int128)(rem - k + 1) / (unsigned __int128)k;
          else
            cl = cl * (long double)(rem - k + 1) / (long double)k;
        }
        const double r = rem <= 125 ? std::sqrt((double)c) : (double)std::sqrt(cl);
        wt[(size_t)rem * V + k] = make_double2(r, 1.0 / r);
      }
    }
    // after the table: the per-N centring powers of two (Tables::wscale)
    for (int N = 0; N < V; ++N) {
      const int e = (int)std::floor(0.5 * log2_max_ket_weight(s.M, N) + 0.5);
      wt.push_back(make_double2(std::ldexp(1.0, -e), std::ldexp(1.0, e)));
    }
    QB_CUDA(cudaMalloc(&s.d_wtab, sizeof(double2) * wt.size()));
    QB_CUDA(cudaMemcpy(s.d_wtab, wt.data(), sizeof(double2) * wt.size(), cudaMemcpyHostToDevice));
    t.wtab = s.d_wtab;
    t.wscale = s.d_wtab + (size_t)V * V;
  }
  {
    const size_t smem = row_smem(t);
    int grid = 0;
    int rc = persistent_grid(diag_kernel, smem, t.total, &grid);
    if (rc) return rc;
    diag_kernel<<<grid, kBlock, smem>>>(t, s.d_diag, s.d_occ, s.d_wi);
    QB_CUDA(cudaGetLastError());
    QB_CUDA(cudaDeviceSynchronize());
  }
  return QB_OK;
}

// workspace: two double-float stage vectors and the double-float copy of psi,
// each [batch][total] x 16 bytes
int64_t workspace_bytes(const Space& s, int batch) { return 3 * (int64_t)batch * s.secOff.back() * 16; }

template <int MODE, int B, bool CPLX>
static int launch_stage(const Space& s, const StageArgs& a, cudaStream_t st, int* grid_out = nullptr) {
  auto k = hpsi_kernel<MODE, B, CPLX>;
  const size_t smem = row_smem(s.t);
  int grid = 0;
  int rc = persistent_grid(k, smem, s.t.total, &grid);
  if (rc) return rc;
  if (grid_out) *grid_out = grid;
  k<<<grid, kBlock, smem, st>>>(s.t, a);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

template <int MODE, int B>
static int launch_stage_c(const Space& s, const StageArgs& a, cudaStream_t st, int* grid_out = nullptr) {
  return s.t.is_complex ? launch_stage<MODE, B, true>(s, a, st, grid_out)
                        : launch_stage<MODE, B, false>(s, a, st, grid_out);
}

int launch_hpsi(const Space& s, const void* d_v, void* d_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  StageArgs a{};
  a.vin = (const double2*)d_v;
  a.out = (double2*)d_out;
  a.scale[0] = 1.0;
  a.status = reinterpret_cast<int*>(s.d_scratch);
  int rc = launch_stage_c<MODE_HPSI, 1>(s, a, st);
  if (rc) return rc;
  return check_status(s, st);
}

// plain = true: one launch per sector per stage (the comparison baseline of
// qb_evolve_plain); otherwise one launch per stage covers every sector.
// Steps are issued one launch per stage for every sector (plain = false) or one
// launch per sector per stage (plain = true, the comparison baseline of
// qb_evolve_plain).  The batched path captures chunks of kGraphSteps steps into
// a CUDA graph once the first step has run (and the launch geometry is cached),
// and replays the graph; a capture that the runtime refuses falls back to issuing
// the launches directly.
constexpr int64_t kGraphSteps = 32;

template <int B>
static int rk4_issue(Space& s, DfArgs& a, double dt, int64_t steps, float4* w1, float4* w2, float4* psif,
                     cudaStream_t st, bool plain, int64_t row0 = 0) {
  const bool cplx = s.t.is_complex != 0;
  const int K = s.order;
  for (int64_t it = 0; it < steps; ++it) {
    // Horner (order K = 4): v = psi + z/4 H psi; v = psi + z/3 H v; v = psi + z/2 H v;
    // psi = psi + z H v; stage j of K reads the previous output and writes w1 / w2
    // alternately, the last one the weighted copy of psi
    for (int d = K; d >= 1; --d) {
      const int j = K - d;
      a.vin = (j == 0) ? psif : ((j - 1) % 2 == 0 ? w1 : w2);
      a.out = (d == 1) ? psif : (j % 2 == 0 ? w1 : w2);
      a.zre = dt / d;
      const float zh = (float)a.zre;
      a.zf = make_float2(zh, (float)(a.zre - (double)zh));
      if (!plain) {
        a.row0 = row0;
        a.row1 = s.t.total;
        int rc = stage_launch(s.t, a, d == 1 ? 1 : 0, B, cplx, st, nullptr, false, s.tile_shape);
        if (rc) return rc;
      } else {
        for (size_t sec = 0; sec + 1 < s.secOff.size(); ++sec) {
          a.row0 = s.secOff[sec];
          a.row1 = s.secOff[sec + 1];
          int rc = stage_launch(s.t, a, d == 1 ? 1 : 0, B, cplx, st, nullptr, false, s.tile_shape);
          if (rc) return rc;
        }
      }
    }
  }
  return QB_OK;
}

template <int B>
static int rk4_loop(Space& s, double2* psi, const double* scale, double dt, int64_t steps, float4* w1, float4* w2,
                    float4* psif, cudaStream_t st, bool plain = false) {
  {
    // the stages run in the weighted basis f = psi / w
    int rc = launch_to_dfw(s, psi, psif, B, st);
    if (rc) return rc;
  }
  DfArgs a{};
  for (int b = 0; b < B; ++b) {
    const float h = (float)scale[b];
    a.scale[b] = make_float2(h, (float)(scale[b] - (double)h));
  }
  a.diag = s.d_diag;
  a.psi = psi;
  a.psif = psif;
  a.status = reinterpret_cast<int*>(s.d_scratch);
  a.nbasef = 0;
  if (plain) return rk4_issue<B>(s, a, dt, steps, w1, w2, psif, st, true);
  // Leading sectors small enough to sit in shared memory run resident on a side
  // stream, all steps in one launch, while the rest advances stage by stage.
  int64_t row0 = 0;
  bool forked = false;
  if (B == 1) {
    int n_small = 0;
    const int nsec = (int)s.secDim.size();
    int optin = 0;
    QB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s.device));
    const size_t base_smem = resident_smem(s.t, 0);
    const int64_t room = optin > (int)base_smem ? (optin - (int64_t)base_smem - 1024) / 64 : 0;
    const int64_t limit = std::min<int64_t>(room, s.resident_max_kets);
    int cap = 0;
    while (n_small < nsec && s.secDim[n_small] <= limit) cap = std::max<int>(cap, (int)s.secDim[n_small++]);
    if (n_small > 0) {
      if (!s.side_stream) QB_CUDA(cudaStreamCreateWithFlags(&s.side_stream, cudaStreamNonBlocking));
      if (!s.ev_fork) QB_CUDA(cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming));
      if (!s.ev_join) QB_CUDA(cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming));
      QB_CUDA(cudaEventRecord(s.ev_fork, st));
      QB_CUDA(cudaStreamWaitEvent(s.side_stream, s.ev_fork, 0));
      ResArgs r{};
      r.psi = psi;
      r.psif = psif;
      r.diag = s.d_diag;
      r.scale = a.scale[0];
      r.dt = dt;
      r.steps = steps;
      r.order = s.order;
      r.n_small = n_small;
      r.cap = cap;
      r.status = a.status;
      int rc = resident_launch(s.t, r, s.t.is_complex != 0, s.side_stream);
      if (rc) return rc;
      QB_CUDA(cudaEventRecord(s.ev_join, s.side_stream));
      forked = true;
      row0 = s.secOff[n_small];
    }
  }
  auto join = [&]() -> int {
    if (forked) QB_CUDA(cudaStreamWaitEvent(st, s.ev_join, 0));
    return QB_OK;
  };
  if (row0 >= s.t.total) return join();
  if (steps < 2 * kGraphSteps) {
    int rc = rk4_issue<B>(s, a, dt, steps, w1, w2, psif, st, false, row0);
    if (rc) return rc;
    return join();
  }
  // first step directly: fills the launch-geometry cache outside any capture
  int rc = rk4_issue<B>(s, a, dt, 1, w1, w2, psif, st, false, row0);
  if (rc) return rc;
  int64_t left = steps - 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool captured = false;
  // capture on the space's private stream (the caller's may be the legacy default
  // stream, which cannot capture); the graph is launched on the caller's stream
  if (!s.capture_stream) QB_CUDA(cudaStreamCreateWithFlags(&s.capture_stream, cudaStreamNonBlocking));
  if (cudaStreamBeginCapture(s.capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    rc = rk4_issue<B>(s, a, dt, kGraphSteps, w1, w2, psif, s.capture_stream, false, row0);
    const cudaError_t ec = cudaStreamEndCapture(s.capture_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) captured = true;
  }
  cudaGetLastError();  // a refused capture leaves a sticky-free error; clear it
  if (captured) {
    for (; left >= kGraphSteps; left -= kGraphSteps) {
      const cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(QB_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
      }
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
  } else if (graph) {
    cudaGraphDestroy(graph);
  }
  rc = rk4_issue<B>(s, a, dt, left, w1, w2, psif, st, false, row0);
  if (rc) return rc;
  return join();
}

int launch_rk4(Space& s, void* d_psi, int batch, const double* scale, double dt, int64_t steps, void* d_work,
               void* stream, bool plain) {
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = (int64_t)batch * s.secOff.back();
  double2* psi = (double2*)d_psi;
  float4* w1 = (float4*)d_work;
  float4* w2 = w1 + n;
  float4* psif = w2 + n;
  int rc;
  switch (batch) {
    case 1: rc = rk4_loop<1>(s, psi, scale, dt, steps, w1, w2, psif, st, plain); break;
    case 2: rc = rk4_loop<2>(s, psi, scale, dt, steps, w1, w2, psif, st, plain); break;
    case 4: rc = rk4_loop<4>(s, psi, scale, dt, steps, w1, w2, psif, st, plain); break;
    case 8: rc = rk4_loop<8>(s, psi, scale, dt, steps, w1, w2, psif, st, plain); break;
    default: return fail(QB_EINVAL, "batch must be 1, 2, 4 or 8");
  }
  if (rc) return rc;
  return check_status(s, st);
}

int launch_to_dfw(const Space& s, const void* psi, void* psif, int B, void* stream) {
  int dev = 0, sms = 0;
  QB_CUDA(cudaGetDevice(&dev));
  QB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = (s.t.total + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  auto k = to_dfw_kernel<0>;
  switch (s.M) {
    case 5: k = to_dfw_kernel<5>; break;
    case 7: k = to_dfw_kernel<7>; break;
    case 9: k = to_dfw_kernel<9>; break;
    case 11: k = to_dfw_kernel<11>; break;
    default: break;
  }
  k<<<grid, 256, 0, (cudaStream_t)stream>>>(s.t, (const double2*)psi, (float4*)psif, B);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

int launch_to_df(const void* psi, void* psif, int64_t n, void* stream) {
  to_df_kernel<<<1216, 256, 0, (cudaStream_t)stream>>>((const double2*)psi, (float4*)psif, n);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

int launch_unrank(const Space& s, int64_t first, int64_t count, int* d_occ, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = row_smem(s.t);
  int grid = 0;
  int rc = persistent_grid(unrank_kernel, smem, count, &grid);
  if (rc) return rc;
  unrank_kernel<<<grid, kBlock, smem, st>>>(s.t, first, count, d_occ, reinterpret_cast<int*>(s.d_scratch));
  QB_CUDA(cudaGetLastError());
  return check_status(s, st);
}

int launch_rank(const Space& s, const int* d_occ, int64_t count, int64_t* d_index, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = blob_smem(s.t);
  int grid = 0;
  int rc = persistent_grid(rank_kernel, smem, count, &grid);
  if (rc) return rc;
  rank_kernel<<<grid, kBlock, smem, st>>>(s.t, d_occ, count, d_index);
  QB_CUDA(cudaGetLastError());
  QB_CUDA(cudaStreamSynchronize(st));
  return QB_OK;
}

int launch_terms(const Space& s, int64_t* terms, int64_t* tuples, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = row_smem(s.t);
  int grid = 0;
  int rc = persistent_grid(terms_kernel, smem, s.t.total, &grid);
  if (rc) return rc;
  unsigned long long* d = reinterpret_cast<unsigned long long*>(partial_area(s));
  QB_CUDA(cudaMemsetAsync(d, 0, 16, st));
  terms_kernel<<<grid, kBlock, smem, st>>>(s.t, d);
  QB_CUDA(cudaGetLastError());
  unsigned long long h[2];
  QB_CUDA(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  *terms = (int64_t)h[0];
  if (tuples) *tuples = (int64_t)h[1];
  return QB_OK;
}

int launch_init_table(const Space& s, const double* table_host, int only_N, void* d_psi, double* norm2,
                      void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = row_smem(s.t);
  int grid = 0;
  int rc = persistent_grid(init_table_kernel, smem, s.t.total, &grid);
  if (rc) return rc;
  double* part = partial_area(s);
  double* tab = table_area(s);
  const size_t tab_bytes = sizeof(double) * 2 * (size_t)s.M * (s.nmax + 1);
  QB_CUDA(cudaMemcpyAsync(tab, table_host, tab_bytes, cudaMemcpyHostToDevice, st));
  init_table_kernel<<<grid, kBlock, smem, st>>>(s.t, (const double2*)tab, only_N, (double2*)d_psi, part);
  QB_CUDA(cudaGetLastError());
  double* fin = init_final(s);
  reduce_partials_kernel<<<1, 32, 0, st>>>(part, grid, 1, fin);
  QB_CUDA(cudaGetLastError());
  QB_CUDA(cudaMemcpyAsync(norm2, fin, sizeof(double), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  return QB_OK;
}

int launch_scale(const Space& s, void* d_psi, double factor, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  scale_kernel<<<1216, 256, 0, st>>>((double2*)d_psi, s.t.total, factor);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

int launch_number(const Space& s, int64_t index, void* d_psi, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  number_kernel<<<1216, 256, 0, st>>>((double2*)d_psi, s.t.total, index);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

// ----------------------------------------------- allocation-free observables
//
// qb_observables_noalloc serves callers that must not allocate device memory
// while they run: code inside a memory-budgeted service or a custom allocator
// that forbids cudaMalloc / cudaFree after start-up, or a host thread that must
// not touch the allocator (which may synchronise the device).  It computes the
// same observables as qb_observables, but its reduction partials live in one
// fixed, file-scope device array instead of the space's scratch buffer.
//
// The array holds kNoAllocDoubles doubles (1 MiB) on every GPU that loads the
// library, for the life of the process.  Every call shares it and it keeps the
// last call's contents; the status word is cleared at the start of each call.
// Calls that overlap on the GPU (several streams or threads at once) race on it.
// The first call on each device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call before
// any stream capture.  The address is cached per device for the process: one CUDA
// context per device for the life of the process is assumed (a cudaDeviceReset
// would reload the module and leave the cached address stale).

constexpr int64_t kNoAllocDoubles = 131072;  // 1 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
static double* g_noalloc_ptr[256];  // device address of the array, per device
static std::mutex g_noalloc_mu;

static int noalloc_scratch(double** out) {
  int dev = 0;
  QB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(QB_EUNSUPPORTED, "device ordinal beyond 255");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(QB_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return QB_OK;
}

// <psi|H psi> partials of at most `grid` CTAs (the size the fixed array was carved
// for); *launched receives the CTA count, the number of partials to reduce
template <bool CPLX>
static int noalloc_dot(const Space& s, const StageArgs& a, int grid, cudaStream_t st, int* launched) {
  const size_t smem = row_smem(s.t);
  auto k = hpsi_kernel<MODE_DOT, 1, CPLX>;
  int g0 = 0;
  int rc = persistent_grid(k, smem, s.t.total, &g0);
  if (rc) return rc;
  *launched = std::min(grid, g0);
  k<<<*launched, kBlock, smem, st>>>(s.t, a);
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

}  // namespace qb

using namespace qb;

extern "C" int qb_observables_noalloc(qb_space* space, const void* d_psi, qb_obs* out, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !out) return fail(QB_EINVAL, "space and out must be non-NULL");
  if (!d_psi || (reinterpret_cast<uintptr_t>(d_psi) & 15)) return fail(QB_EINVAL, "d_psi must be 16-byte aligned");
  int dev = 0;
  QB_CUDA(cudaGetDevice(&dev));
  if (dev != sp->device) return fail(QB_EINVAL, "the space was built on another device");
  double* scr = nullptr;
  int rc = noalloc_scratch(&scr);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int M = sp->M;
  const int nmom = nmoments(M);
  // layout (doubles): [0, 2) status word | partials [G nmom] | final [nmom] |
  // dot partials [2 G] | dot final [2]; G CTAs, capped so that it fits
  const int64_t fixed = 2 + nmom + 2 + 8;
  const int64_t gcap = (kNoAllocDoubles - fixed) / (nmom + 2);
  if (gcap < 32)
    return fail(QB_EUNSUPPORTED, "the moments of this space need more than the fixed 1 MiB scratch of "
                                 "qb_observables_noalloc (M too large)");
  const size_t smem = row_smem(sp->t) + ((kRowScratchBytes + 15) & ~15) - kRowScratchBytes +
                      (size_t)(kBlock / 32) * nmom * sizeof(double) + 16;
  int grid = 0;
  rc = persistent_grid(moments_kernel, smem, sp->t.total, &grid);
  if (rc) return rc;
  grid = (int)std::min<int64_t>(grid, gcap);
  int* status = reinterpret_cast<int*>(scr);
  double* part = scr + 2;
  double* fin = part + (int64_t)grid * nmom;
  double* dpart = fin + nmom;
  double* dfin = dpart + 2 * (int64_t)grid;
  QB_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  moments_kernel<<<grid, kBlock, smem, st>>>(sp->t, (const double2*)d_psi, part, nmom, status);
  QB_CUDA(cudaGetLastError());
  reduce_partials_kernel<<<(nmom + 127) / 128, 128, 0, st>>>(part, grid, nmom, fin);
  QB_CUDA(cudaGetLastError());
  StageArgs a{};
  a.vin = (const double2*)d_psi;
  a.scale[0] = 1.0;
  a.status = status;
  a.partial = dpart;
  int gdot = 0;
  rc = sp->t.is_complex ? noalloc_dot<true>(*sp, a, grid, st, &gdot) : noalloc_dot<false>(*sp, a, grid, st, &gdot);
  if (rc) return rc;
  reduce_partials_kernel<<<1, 32, 0, st>>>(dpart, gdot, 2, dfin);
  QB_CUDA(cudaGetLastError());
  std::vector<double> raw(nmom, 0.0);
  double h2[2];
  int hs = 0;
  QB_CUDA(cudaMemcpyAsync(raw.data(), fin, sizeof(double) * nmom, cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaMemcpyAsync(h2, dfin, sizeof(h2), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  if (hs) return fail(QB_EINTERNAL, "device-side consistency check failed (status " + std::to_string(hs) + ")");
  raw[2] = h2[0];
  if (!(raw[0] > 0.0)) return fail(QB_EINVAL, "the state has zero norm");
  derive(M, raw.data(), out);
  return QB_OK;
}

namespace qb {

}  // namespace qb
