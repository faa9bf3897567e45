// Observables of Sec. II C-E on the GPU: the raw moments norm, <N>, <H>, <a_i>,
// <a_i^dag a_j>, <a_i a_j> of one state, with FP64 reductions.
//
// One call runs three kernels over every ket n of the space (amplitude psi_n):
//  1. obs_prep_kernel: the weighted double-float copy f = psi / w of the state (the
//     basis of the RK4 stages, w(n) = sqrt(N! / prod n_m!) 2^-e_N) and the moments
//     that need no other ket: |psi|^2 and N |psi|^2 summed in FP64, n_i |psi|^2 in
//     double-float over 32 kets at a time, added in FP64.
//  2. moments_w_kernel: every moment that moves the ket, conj(psi_t) c psi_n with
//     t = O n for O = a_i, a_i^dag a_j (i < j; the rest by Hermiticity) and a_i a_j
//     (i <= j), gathered from f.  In the weighted basis
//        conj(psi_t) c psi_n = conj(f_t) (psi_n w_n) k 2^(e_N - e_N') / sqrt(N! / N'!)
//     with N' the particle number of t and k a small integer: n_i (a_i), n_j
//     (a_i^dag a_j), n_i n_j or n_i (n_i - 1) (a_i a_j): the square roots of the
//     ladder operators cancel against the ratio of ket weights.
//  3. the double-float stage kernel in its <x|H|x> mode on f, each row's
//     Re(conj(f_n) (W^-1 H W f)_n) multiplied by w_n^2 in FP64.
// Every sum over kets is FP64: per-thread FP64 accumulators in kernels 1 and 3, and
// where a term is a double-float product (n_i |psi|^2 in kernel 1, the gathered
// moments in kernel 2) the products of 32 kets are summed in double-float and each
// such partial is added to an FP64 accumulator.  CTA rows and the sum over CTAs are
// FP64 in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "qb_device.cuh"
#include "qb_internal.h"
#include "qb_stage.cuh"

namespace qb {

constexpr int kObsBlock = 256;  // threads per CTA of the first pass
// warps per CTA of the moments kernel (its CTAs share nothing but the staged table);
// the kernels with two entries a lane keep two kets in flight, which takes more
// registers a thread, and run fewer warps
#ifndef QB_MW_WARPS
#define QB_MW_WARPS 24
#endif
#ifndef QB_MW_WARPS_SPL2
#define QB_MW_WARPS_SPL2 20
#endif
constexpr int kMwSplMax = 3;    // moment entries per lane and pass (<= 96 per pass)
// resident CTAs per SM the moments kernel's registers are planned for
#ifndef QB_MW_MIN_BLOCKS
#define QB_MW_MIN_BLOCKS 1
#endif
// moments kernels with at most two entries a lane keep two kets' gathers in flight
#ifndef QB_MW_PIPE
#define QB_MW_PIPE 1
#endif
__host__ __device__ constexpr int mw_warps(int spl) { return (QB_MW_PIPE && spl == 2) ? QB_MW_WARPS_SPL2 : QB_MW_WARPS; }

// sums partial[0..n)[0..width) over the first index in a fixed order
__global__ void reduce_rows_kernel(const double* partial, int n, int width, double* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < width; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partial[(size_t)k * width + c];
    out[c] = s;
  }
}

// FP64 sum over the CTA in a fixed order: lanes by shuffles, then warps in turn;
// `red` holds one value per warp.  The result is valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // red may still be read by the previous call
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Pass 1: f = df(psi / w) and the FP64 sums of |psi|^2, N |psi|^2, n_i |psi|^2;
// partial[block][nprep(M)].
template <int MT>
__global__ void __launch_bounds__(kObsBlock) obs_prep_kernel(const Tables t, const double2* psi, float4* f,
                                                             double* partial) {
  __shared__ double red[kObsBlock / 32];
  const int M = (MT > 0) ? MT : t.M;
  constexpr int kMB = (MT > 0) ? MT : kMaxM;
  const int ob = t.occ_bits;
  // norm and <N> in FP64 per ket; <n_i> as double-float sums of |psi|^2 n_i over 32
  // kets at a time, each added to an FP64 sum (the FP64 pipe is the limit here)
  double nrm = 0.0, nN = 0.0, ni[kMB];
  dfl nt[kMB];
#pragma unroll
  for (int m = 0; m < kMB; ++m) {
    ni[m] = 0.0;
    nt[m] = dfl{0.f, 0.f};
  }
  int cnt = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < t.total; g += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t word = __ldg(t.occ + g);
    const double2 x = psi[g];
    const double wi = __ldg(t.wi + g);
    f[g] = df_pack(df_of(x.x * wi), df_of(x.y * wi));
    const double p2 = x.x * x.x + x.y * x.y;
    const dfl p2f = df_of(p2);
    int N = 0;
#pragma unroll
    for (int m = 0; m < kMB; ++m)
      if (m < M) {
        const int nm = occ_of(word, m, ob);
        N += nm;
        nt[m] = df_add(nt[m], df_mul_f(p2f, (float)nm));
      }
    nrm += p2;
    nN += p2 * (double)N;
    if (++cnt == 32) {
      cnt = 0;
#pragma unroll
      for (int m = 0; m < kMB; ++m)
        if (m < M) {
          ni[m] += df_to(nt[m]);
          nt[m] = dfl{0.f, 0.f};
        }
    }
  }
#pragma unroll
  for (int m = 0; m < kMB; ++m)
    if (m < M) ni[m] += df_to(nt[m]);
  const int w = nprep(M);
  double s = cta_sum(nrm, red);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * w] = s;
  s = cta_sum(nN, red);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * w + 1] = s;
#pragma unroll
  for (int m = 0; m < kMB; ++m)
    if (m < M) {
      s = cta_sum(ni[m], red);
      if (threadIdx.x == 0) partial[(size_t)blockIdx.x * w + 2 + m] = s;
    }
}

// ---------------------------------------------------------------- moment entries
//
// Entry s of the moments kernel: [0, M) a_i; then a_i^dag a_j for i < j (the ket
// loses one particle in j and gains one in i); then a_i a_j for i <= j.  The target
// ket changes mode e0 by dn0 and mode e1 by dn1; k = n_e0 (times n_e1 + c1 when the
// entry has a second factor); the class picks the scale of the target's particle
// number: 0 same N, 1 N - 1, 2 N - 2.
enum { kEntA = 0, kEntAdA = 1, kEntAA = 2 };

__host__ __device__ inline int mw_entries(int M) { return M + M * (M - 1) / 2 + M * (M + 1) / 2; }

struct MwEntry {
  int kind, i, j;         // the operator: a_i, a_i^dag a_j or a_i a_j
  int e0, dn0, e1, dn1;   // occupation changes of the target
  int has2, c1, cls;      // k = n_e0 (n_e1 + c1 if has2); class of the scale
};

__host__ __device__ inline MwEntry mw_entry(int s, int M) {
  MwEntry e{};
  if (s < M) {
    e.kind = kEntA;
    e.i = e.j = s;
    e.e0 = e.e1 = s;
    e.dn0 = -1;
    e.cls = 1;
    return e;
  }
  s -= M;
  int i = 0;
  if (s < M * (M - 1) / 2) {
    while (s >= M - 1 - i) {
      s -= M - 1 - i;
      ++i;
    }
    e.kind = kEntAdA;
    e.i = i;
    e.j = i + 1 + s;
    e.e0 = e.j;  // annihilate j
    e.dn0 = -1;
    e.e1 = e.i;  // create i
    e.dn1 = 1;
    e.cls = 0;
    return e;
  }
  s -= M * (M - 1) / 2;
  while (s >= M - i) {
    s -= M - i;
    ++i;
  }
  e.kind = kEntAA;
  e.i = i;
  e.j = i + s;
  e.cls = 2;
  e.has2 = 1;
  e.e0 = e.i;
  if (e.i == e.j) {  // n_i (n_i - 1)
    e.dn0 = -2;
    e.e1 = e.i;
    e.c1 = -1;
  } else {  // n_i n_j
    e.dn0 = -1;
    e.e1 = e.j;
    e.dn1 = -1;
  }
  return e;
}

// shared memory of moments_w_kernel after the staged ranking table (all 16-byte
// multiples): entry headers [np] int4, byte shifts [iwords][np] int32, class scales
// [3][nmax+1] float2, the CTA's FP64 moment row [nmom], and per warp the staged
// tile of 32 kets (x float4, occupations as bytes [obwords] uint32, (N, K) int32,
// offsets [iwords] int32)
__host__ __device__ inline size_t mw_smem_after(int np, int nmax, int nmom, int iwords, int obwords, int warps) {
  return (size_t)np * 16 + (((size_t)iwords * np * 4 + 15) & ~(size_t)15) +
         ((3 * (size_t)(nmax + 1) * 8 + 15) & ~(size_t)15) + (((size_t)nmom * 8 + 15) & ~(size_t)15) +
         (size_t)warps * 32 * (16 + 4 * (size_t)obwords + 4 + 4 * (size_t)iwords);
}

// n_m from occupations packed as bytes, four modes a word (M <= 16): one byte
// permute of the two words that hold mode m
template <int NW>
__device__ __forceinline__ int mw_occ(const uint32_t (&w)[NW], int m) {
  if constexpr (NW <= 2) {
    return (int)(__byte_perm(w[0], NW > 1 ? w[NW - 1] : 0u, (uint32_t)m) & 0xffu);
  } else {
    const bool hi = m >= 8;
    const uint32_t x = hi ? w[2] : w[0];
    const uint32_t y = hi ? (NW > 3 ? w[NW - 1] : 0u) : w[1];
    return (int)(__byte_perm(x, y, (uint32_t)(m & 7)) & 0xffu);
  }
}

// bytes of the ranking table (16-byte multiple: the next table starts aligned)
__host__ __device__ inline int mw_table_bytes(const Tables& t) { return t.o_ann - t.o_E; }

constexpr size_t kMwSecSmemMax = 16384;  // sector tables larger than this stay in global memory

static size_t mw_sec_bytes(const Tables& t) {
  return ((sizeof(int64_t) * (size_t)(t.n_sectors + 1) + 15) & ~(size_t)15) +
         ((sizeof(int32_t) * (size_t)(t.nmax + 1) * t.Q + 15) & ~(size_t)15);
}

__device__ __forceinline__ int find_sector_in(const int64_t* off, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// x mod Q for x in (-2Q, 3Q), by conditional adds
__device__ __forceinline__ int mod_small(int x, int Q) {
  if (x < 0) x += Q;
  if (x < 0) x += Q;
  if (x >= Q) x -= Q;
  if (x >= Q) x -= Q;
  return x;
}

// Pass 2: the moments that move the ket, entries [e_begin, e_begin + nent) of this
// pass (nent <= 32 kMwSpl).  The lanes of a warp take the entries (kMwSpl per lane);
// the 32 kets of a tile are staged in the warp's shared memory -- x = psi_n w_n
// (double-float), the packed occupations, (N, K) and the suffix-state offsets of the
// ranking table -- and visited in turn, every lane reading ket j's data by broadcast.
// A target's rank is D - 1 - sum_{m=1}^{M-1} E[idx_m + shift_m], the shift of the
// suffix index at mode m depending only on the entry; for momentum mod M the byte
// offsets of two modes share a 32-bit word (as in the stage kernel), for exact
// momentum each mode has its own.  partial[block][nmom] (FP64).
template <int MT, bool EXACT>
struct MwWords {  // 32-bit words of suffix-state offsets per ket
  static constexpr int n = EXACT ? ((MT > 0) ? MT : kMaxM) : ((MT > 0) ? (MT / 2 > 0 ? MT / 2 : 1) : kMaxM / 2);
};
template <int MT>
struct MwOccWords {  // 32-bit words of byte occupations per ket
  static constexpr int n = (MT > 0) ? (MT + 3) / 4 : kMaxM / 4;
};

template <int MT, bool EXACT, int kMwSpl>
__global__ void __launch_bounds__(32 * mw_warps(kMwSpl), QB_MW_MIN_BLOCKS) moments_w_kernel(const Tables t, const double2* psi, const float4* f,
                                                                 double* partial, int nmom, int e_begin, int nent,
                                                                 int sec_smem, int* status, const float4* ketf,
                                                                 const int* tb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kMwWarps = mw_warps(kMwSpl), kMwBlock = 32 * kMwWarps;
  constexpr int kMB = (MT > 0) ? MT : kMaxM;
  constexpr int kIW = MwWords<MT, EXACT>::n;
  constexpr int kOBW = MwOccWords<MT>::n;
  // shared memory starts with the ranking table (mod M; exact momentum keeps it in
  // global memory and stages nothing)
  const int e_bytes = EXACT ? 0 : mw_table_bytes(t);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = (MT > 0) ? MT : t.M, Q = t.Q, twoQ = 2 * Q, V = t.nmax + 1;
  const int np = (nent + 31) & ~31;
  const int iw = EXACT ? M : M / 2;  // offset words in use (mode m: word m, or word (m-1)/2 packed)
  unsigned char* cur = smem_raw + e_bytes;
  int4* hdr = reinterpret_cast<int4*>(cur);  // e0 | e1 << 8 | has2 << 16 | cls << 24, c1, dN, dK mod Q
  cur += (size_t)np * 16;
  int32_t* shf = reinterpret_cast<int32_t*>(cur);  // [kIW][np] byte shifts (packed in pairs for mod M)
  cur += ((size_t)kIW * np * 4 + 15) & ~(size_t)15;
  float2* scl = reinterpret_cast<float2*>(cur);  // [3][V] double-float scale of each class at particle number N
  cur += (3 * (size_t)V * 8 + 15) & ~(size_t)15;
  double* row = reinterpret_cast<double*>(cur);  // [nmom]
  cur += ((size_t)nmom * 8 + 15) & ~(size_t)15;
  // per warp: the tile's kets (x, occupations, (N, K), offset words)
  float4* kx = reinterpret_cast<float4*>(cur) + (size_t)warp * 32;
  cur += (size_t)kMwWarps * 32 * 16;
  uint32_t* kob = reinterpret_cast<uint32_t*>(cur) + (size_t)warp * 32 * kOBW;  // [kOBW][32]
  cur += (size_t)kMwWarps * 32 * kOBW * 4;
  int32_t* knk = reinterpret_cast<int32_t*>(cur) + (size_t)warp * 32;
  cur += (size_t)kMwWarps * 32 * 4;
  int32_t* kid = reinterpret_cast<int32_t*>(cur) + (size_t)warp * 32 * kIW;  // [kIW][32]
  cur += (size_t)kMwWarps * 32 * kIW * 4;
  for (int s = tid; s < np; s += kMwBlock) {
    int4 h = make_int4(0, 0, 0, 0);
    int sh[kMaxM];
    for (int m = 0; m < kMaxM; ++m) sh[m] = 0;
    if (s < nent && tb) {
      // two-body operator a_a1^dag a_a2^dag a_c1 a_c2 (tb[] = a1 | a2 << 8 | c1 << 16 | c2 << 24):
      // k = n_c1 (n_c2 - [c1 = c2]), the target in the same sector; the suffix shift
      // of mode m sums the changes of the modes >= m
      const int w = tb[e_begin + s];
      const int a1 = w & 0xff, a2 = (w >> 8) & 0xff, c1 = (w >> 16) & 0xff, c2 = (w >> 24) & 0xff;
      int dc = 0, dk = 0;
      for (int m = M - 1; m >= 1; --m) {
        const int dm = (m == a1) + (m == a2) - (m == c1) - (m == c2);
        dc += dm;
        dk += dm * m;
        sh[m] = dc * twoQ + (((dk % Q) + Q) % Q);
      }
      h = make_int4(c1 | (c2 << 8) | (1 << 16), c1 == c2 ? -1 : 0, 0, 0);
    } else if (s < nent) {
      const MwEntry e = mw_entry(e_begin + s, M);
      const int f1 = (e.dn1 == 0) ? e.e0 : e.e1;  // a zero second change acts on e0
      const int hi = max(e.e0, f1), lo = min(e.e0, f1);
      const int dh = (hi == e.e0) ? e.dn0 : e.dn1;
      const int shh = dh * twoQ + mod_small(dh * hi, Q);
      const int dc = e.dn0 + e.dn1, dk = mod_small(e.dn0 * e.e0 + e.dn1 * f1, Q);
      for (int m = 1; m < M; ++m) sh[m] = m > hi ? 0 : (m > lo ? shh : dc * twoQ + dk);
      h = make_int4(e.e0 | (e.e1 << 8) | (e.has2 << 16) | (e.cls << 24), e.c1, dc, dk);
    }
    hdr[s] = h;
    for (int k = 0; k < kIW; ++k) {
      int v = 0;
      if (EXACT) {
        if (k >= 1 && k < M) v = 4 * sh[k];
      } else if (2 * k + 1 < M) {  // signed lo + 65536 hi, so that the low half's borrow is part of it
        v = 4 * sh[2 * k + 1] + 65536 * 4 * ((2 * k + 2 < M) ? sh[2 * k + 2] : 0);
      }
      shf[k * np + s] = v;
    }
  }
  // class scales: 1, 2^(e_N - e_{N-1}) / sqrt(N), 2^(e_N - e_{N-2}) / sqrt(N (N - 1))
  for (int k = tid; k < 3 * V; k += kMwBlock) {
    const int c = k / V, N = k % V;
    double v = 1.0;
    if (c == 1) v = (N >= 1) ? __ldg(t.wscale + N).y * __ldg(t.wscale + N - 1).x / sqrt((double)N) : 0.0;
    if (c == 2) v = (N >= 2) ? __ldg(t.wscale + N).y * __ldg(t.wscale + N - 2).x / sqrt((double)N * (N - 1)) : 0.0;
    const dfl d = df_of(v);
    scl[k] = make_float2(d.h, d.l);
  }
  const int64_t* soff = t.sec_off;
  const int32_t* sof = t.sec_of;
  if (sec_smem) {
    int64_t* o = reinterpret_cast<int64_t*>(cur);
    for (int k = tid; k <= t.n_sectors; k += kMwBlock) o[k] = __ldg(t.sec_off + k);
    cur += (sizeof(int64_t) * (size_t)(t.n_sectors + 1) + 15) & ~(size_t)15;
    int32_t* q = reinterpret_cast<int32_t*>(cur);
    for (int k = tid; k < (t.nmax + 1) * Q; k += kMwBlock) q[k] = __ldg(t.sec_of + k);
    soff = o;
    sof = q;
  }
  for (int k = tid; k < nmom; k += kMwBlock) row[k] = 0.0;
  {
    const int4* src = reinterpret_cast<const int4*>(t.blob + t.o_E);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    for (int i = tid; i < e_bytes / 16; i += kMwBlock) dst[i] = __ldg(src + i);
    __syncthreads();
  }
  const char* Eg = reinterpret_cast<const char*>(t.blob + t.o_E);  // exact momentum: the table stays global
  const int ob = t.occ_bits;
  const int64_t total = t.total;
  const int64_t ntiles = (total + 31) / 32;
  const int rem_w = t.rem_w;

  // this lane's entries in registers for the whole sweep: the modes whose
  // occupations form k (e0 | e1 << 8 | has2 << 16 | (c1 = -1) << 17), and, where
  // the registers allow, the byte shifts of the target's suffix indices
  constexpr bool kHoist = kMwSpl * (1 + kIW) <= 10;
  uint32_t mop[kMwSpl];
  uint32_t msh[kMwSpl][kHoist ? kIW : 1];
#pragma unroll
  for (int r = 0; r < kMwSpl; ++r) {
    const int s = min(r * 32 + lane, np - 1);
    const int4 h = hdr[s];
    mop[r] = (uint32_t)(h.x & 0x1ffff) | (h.y != 0 ? 1u << 17 : 0u);
#pragma unroll
    for (int q = 0; q < (kHoist ? kIW : 1); ++q) msh[r][q] = kHoist ? (uint32_t)shf[q * np + s] : 0u;
  }

  int cur_nk = -1;
  int64_t toff[kMwSpl];
  int tD[kMwSpl];
  dfl csc[kMwSpl];  // class scale at the current N
  double acc_r[kMwSpl], acc_i[kMwSpl];
#pragma unroll
  for (int r = 0; r < kMwSpl; ++r) {
    toff[r] = 0;
    tD[r] = -1;
    csc[r] = dfl{0.f, 0.f};
    acc_r[r] = acc_i[r] = 0.0;
  }

  for (int64_t tile = (int64_t)blockIdx.x * kMwWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kMwWarps) {
    {  // stage this lane's ket: x = psi w (double-float), occupations as bytes, (N, K), offsets
      const int64_t g = tile * 32 + lane;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      uint32_t obw[kOBW];
#pragma unroll
      for (int k = 0; k < kOBW; ++k) obw[k] = 0u;
      int nk = 0;
      uint32_t pk[kIW];
#pragma unroll
      for (int k = 0; k < kIW; ++k) pk[k] = 0u;
      if (g < total) {
        const int sid = find_sector_in(soff, t.n_sectors, g);
        nk = __ldg(t.sec_N + sid) | (__ldg(t.sec_K + sid) << 16);
        const uint64_t word = __ldg(t.occ + g);
        const double w = ket_weight_word<MT>(t, word).x;
        if (tb) {  // a weighted double-float ket k: true value w k, times w
          const float4 kv = ketf[g];
          const double w2 = w * w;
          x = df_pack(df_of(df_to(df_re(kv)) * w2), df_of(df_to(df_im(kv)) * w2));
        } else {
          const double2 p = psi[g];
          x = df_pack(df_of(p.x * w), df_of(p.y * w));
        }
        int srem = 0, skr = 0;
#pragma unroll
        for (int m = kMB - 1; m >= 0; --m) {
          if (m < M) {
            const int nm = occ_of(word, m, ob);
            obw[m >> 2] |= (uint32_t)nm << (8 * (m & 3));
            if (m == 0) continue;
            srem += nm;
            skr += m * nm;
            while (skr >= Q) skr -= Q;
            const uint32_t ix4 = 4u * (uint32_t)((m * rem_w + srem + 2) * twoQ + skr);
#pragma unroll
            for (int k = 0; k < kIW; ++k) {
              if (EXACT) {
                if (k == m) pk[k] = ix4;
              } else if (k == ((m - 1) >> 1)) {
                pk[k] |= ix4 << ((m & 1) ? 0 : 16);
              }
            }
          }
        }
      }
      __syncwarp();  // the previous tile's reads are done
      kx[lane] = x;
#pragma unroll
      for (int k = 0; k < kOBW; ++k) kob[k * 32 + lane] = obw[k];
      knk[lane] = nk;
#pragma unroll
      for (int k = 0; k < kIW; ++k) kid[k * 32 + lane] = (int32_t)pk[k];
      __syncwarp();
    }
    // products of this tile, double-float, (re, im) packed
    dfc tp[kMwSpl];
#pragma unroll
    for (int r = 0; r < kMwSpl; ++r) tp[r] = dfc{0ull, 0ull};
    const int nt = (int)min((int64_t)32, total - tile * 32);
#if QB_MW_PIPE
    if constexpr (kMwSpl <= 2) {
      // two kets in flight: the targets of ket j + 1 are ranked and gathered before
      // the products of ket j, which keeps twice the gathers outstanding per warp.
      // issue(j): the coefficient c = k scale(N) (0 where the operator annihilates
      // the ket or has no target sector) and the gathered target y of each entry
      auto issue = [&](int j, float4 (&y)[kMwSpl], dfl (&cc)[kMwSpl]) {
        const int nkj = knk[j];
        if (nkj != cur_nk) {  // warp-uniform: a new (N, K) sector
          cur_nk = nkj;
          const int N = nkj & 0xffff, K = nkj >> 16;
#pragma unroll
          for (int r = 0; r < kMwSpl; ++r) {
            tD[r] = -1;
            const int s = r * 32 + lane;
            if (s >= nent) continue;
            const int4 h = hdr[s];
            const int Nt = N + h.z;
            if (Nt < 0) continue;
            int Kt = K + h.w;
            if (Kt >= Q) Kt -= Q;
            const int sid = sof[Nt * Q + Kt];
            if (sid < 0) continue;
            toff[r] = soff[sid];
            tD[r] = (int)(soff[sid + 1] - toff[r]);
            const float2 c = scl[((h.x >> 24) & 3) * V + N];
            csc[r] = dfl{c.x, c.y};
          }
        }
        uint32_t obj[kOBW];
#pragma unroll
        for (int k = 0; k < kOBW; ++k) obj[k] = kob[k * 32 + j];
        int idj[kIW];
#pragma unroll
        for (int q = 0; q < kIW; ++q) idj[q] = kid[q * 32 + j];
#pragma unroll
        for (int r = 0; r < kMwSpl; ++r) {
          const uint32_t op = mop[r];
          int k = mw_occ<kOBW>(obj, (int)(op & 0xffu));
          if (op & 0x10000u) k *= mw_occ<kOBW>(obj, (int)((op >> 8) & 0xffu)) - (int)((op >> 17) & 1u);
          bool act = k > 0 && tD[r] >= 0;
          y[r] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (act) {
            int esum = 0;
#pragma unroll
            for (int q = 0; q < kIW; ++q) {
              if (q >= iw) break;
              const uint32_t u =
                  (uint32_t)idj[q] + (kHoist ? msh[r][kHoist ? q : 0] : (uint32_t)shf[q * np + r * 32 + lane]);
              if (EXACT) {
                if (q >= 1) esum += *reinterpret_cast<const int32_t*>(Eg + u);
              } else {
                esum += e_byte(u & 0xffffu);
                if (MT == 0 || 2 * q + 2 < MT) esum += e_byte(u >> 16);
              }
            }
            const int rk = tD[r] - 1 - esum;
            if ((unsigned)rk >= (unsigned)tD[r]) {
              atomicOr(status, 1);
              act = false;
            } else {
              y[r] = __ldg(f + toff[r] + rk);
            }
          }
          cc[r] = df_mul_f(csc[r], act ? (float)k : 0.f);
        }
      };
      // consume(j): tp += c conj(y) x_j, the same arithmetic as the one-ket loop
      auto consume = [&](int j, const float4 (&y4)[kMwSpl], const dfl (&cc)[kMwSpl]) {
        const float4 xj = kx[j];
#pragma unroll
        for (int r = 0; r < kMwSpl; ++r) {
          const float4 y = y4[r];
          const f2 xr = f2_pack(xj.x, xj.x), nxr = f2_pack(-xj.x, -xj.x), xrl = f2_pack(xj.z, xj.z);
          const f2 xi = f2_pack(xj.y, xj.y), nxi = f2_pack(-xj.y, -xj.y), xil = f2_pack(xj.w, xj.w);
          const f2 one_m = f2_pack(1.f, -1.f);
          const f2 Ph = f2_mul(f2_pack(y.x, y.y), one_m), Pl = f2_mul(f2_pack(y.z, y.w), one_m);
          const f2 Sh = f2_pack(y.y, y.x), Sl = f2_pack(y.w, y.z);
          const f2 n1 = f2_mul(nxr, Ph);
          f2 e1 = f2_fma(xr, Ph, n1);
          e1 = f2_fma(xr, Pl, e1);
          e1 = f2_fma(xrl, Ph, e1);
          const f2 n2 = f2_mul(nxi, Sh);
          f2 e2 = f2_fma(xi, Sh, n2);
          e2 = f2_fma(xi, Sl, e2);
          e2 = f2_fma(xil, Sh, e2);
          const f2 ns = f2_add(n1, n2);
          const f2 bb = f2_sub(ns, n1);
          const f2 nerr = f2_add(f2_sub(n1, f2_sub(ns, bb)), f2_sub(n2, bb));
          const f2 nsl = f2_sub(f2_sub(nerr, e1), e2);
          const dfl c = cc[r];
          const f2 Ch = f2_pack(c.h, c.h), nCh = f2_pack(-c.h, -c.h), nCl = f2_pack(-c.l, -c.l);
          dfc_fma(tp[r], nCh, Ch, nCl, ns, nsl);
        }
      };
      float4 ya[kMwSpl], yb[kMwSpl];
      dfl ca[kMwSpl], cb[kMwSpl];
      issue(0, ya, ca);
      for (int j = 0; j < nt; j += 2) {
        const bool two = j + 1 < nt;
        if (two) issue(j + 1, yb, cb);
        consume(j, ya, ca);
        if (two) {
          if (j + 2 < nt) issue(j + 2, ya, ca);
          consume(j + 1, yb, cb);
        }
      }
    } else {
#endif
    for (int j = 0; j < nt; ++j) {
      const int nkj = knk[j];
      if (nkj != cur_nk) {  // warp-uniform: a new (N, K) sector
        cur_nk = nkj;
        const int N = nkj & 0xffff, K = nkj >> 16;
#pragma unroll
        for (int r = 0; r < kMwSpl; ++r) {
          tD[r] = -1;
          const int s = r * 32 + lane;
          if (s >= nent) continue;
          const int4 h = hdr[s];
          const int Nt = N + h.z;
          if (Nt < 0) continue;
          int Kt = K + h.w;
          if (Kt >= Q) Kt -= Q;
          const int sid = sof[Nt * Q + Kt];
          if (sid < 0) continue;  // the target sector is not part of the space
          toff[r] = soff[sid];
          tD[r] = (int)(soff[sid + 1] - toff[r]);
          const float2 c = scl[((h.x >> 24) & 3) * V + N];
          csc[r] = dfl{c.x, c.y};
        }
      }
      const float4 xj = kx[j];
      uint32_t obj[kOBW];
#pragma unroll
      for (int k = 0; k < kOBW; ++k) obj[k] = kob[k * 32 + j];
      // the ket's suffix offsets, read once per ket where the registers allow
      constexpr bool kHoistKet = kMwSpl <= 2;
      int idj[kHoistKet ? kIW : 1];
#pragma unroll
      for (int q = 0; q < (kHoistKet ? kIW : 1); ++q) idj[q] = kHoistKet ? kid[q * 32 + j] : 0;
#pragma unroll
      for (int r = 0; r < kMwSpl; ++r) {
        const uint32_t op = mop[r];
        int k = mw_occ<kOBW>(obj, (int)(op & 0xffu));
        if (op & 0x10000u) k *= mw_occ<kOBW>(obj, (int)((op >> 8) & 0xffu)) - (int)((op >> 17) & 1u);
        // k = 0: the operator annihilates this ket; tD < 0: no target sector
        bool act = k > 0 && tD[r] >= 0;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          int esum = 0;
#pragma unroll
          for (int q = 0; q < kIW; ++q) {
            if (q >= iw) break;
            const uint32_t u = (uint32_t)(kHoistKet ? idj[kHoistKet ? q : 0] : kid[q * 32 + j]) +
                               (kHoist ? msh[r][kHoist ? q : 0] : (uint32_t)shf[q * np + r * 32 + lane]);
            if (EXACT) {
              if (q >= 1) esum += *reinterpret_cast<const int32_t*>(Eg + u);
            } else {
              esum += e_byte(u & 0xffffu);
              // the high half of the last word is mode M when M is even: offset 0 holds zero
              if (MT == 0 || 2 * q + 2 < MT) esum += e_byte(u >> 16);
            }
          }
          const int rk = tD[r] - 1 - esum;
          if ((unsigned)rk >= (unsigned)tD[r]) {
            atomicOr(status, 1);
            act = false;
          } else {
            y = __ldg(f + toff[r] + rk);
          }
        }
        // (three entries a lane: skip instead of adding zeros, which keeps the
        // registers of the unrolled entries apart)
        if (kMwSpl >= 3 && !act) continue;
        // conj(y) x = x_r (y_r, -y_i) + x_i (y_i, y_r), lane 0 the real part
        const f2 xr = f2_pack(xj.x, xj.x), nxr = f2_pack(-xj.x, -xj.x), xrl = f2_pack(xj.z, xj.z);
        const f2 xi = f2_pack(xj.y, xj.y), nxi = f2_pack(-xj.y, -xj.y), xil = f2_pack(xj.w, xj.w);
        const f2 one_m = f2_pack(1.f, -1.f);
        const f2 Ph = f2_mul(f2_pack(y.x, y.y), one_m), Pl = f2_mul(f2_pack(y.z, y.w), one_m);
        const f2 Sh = f2_pack(y.y, y.x), Sl = f2_pack(y.w, y.z);
        // exact products with their error terms
        const f2 n1 = f2_mul(nxr, Ph);
        f2 e1 = f2_fma(xr, Ph, n1);
        e1 = f2_fma(xr, Pl, e1);
        e1 = f2_fma(xrl, Ph, e1);
        const f2 n2 = f2_mul(nxi, Sh);
        f2 e2 = f2_fma(xi, Sh, n2);
        e2 = f2_fma(xi, Sl, e2);
        e2 = f2_fma(xil, Sh, e2);
        // the negated sum -(p1 + p2) = n1 + n2 by TwoSum, ns + nsl with the error terms
        const f2 ns = f2_add(n1, n2);
        const f2 bb = f2_sub(ns, n1);
        const f2 nerr = f2_add(f2_sub(n1, f2_sub(ns, bb)), f2_sub(n2, bb));
        const f2 nsl = f2_sub(f2_sub(nerr, e1), e2);
        // times the coefficient c = k * scale: acc += (-c)(ns + nsl) = c conj(y) x
        const dfl c = df_mul_f(csc[r], act ? (float)k : 0.f);
        const f2 Ch = f2_pack(c.h, c.h), nCh = f2_pack(-c.h, -c.h), nCl = f2_pack(-c.l, -c.l);
        dfc_fma(tp[r], nCh, Ch, nCl, ns, nsl);
      }
    }
#if QB_MW_PIPE
    }
#endif
    // the tile's sums into the lane's FP64 accumulators
#pragma unroll
    for (int r = 0; r < kMwSpl; ++r) {
      float hr, hi2, lr, li;
      f2_unpack(tp[r].h, hr, hi2);
      f2_unpack(tp[r].l, lr, li);
      acc_r[r] += (double)hr + (double)lr;
      acc_i[r] += (double)hi2 + (double)li;
    }
  }
  // the lanes' sums into the CTA's FP64 row, one warp at a time (a fixed order); the
  // entries of a warp land on distinct moments
  const int oA = 4, oM = 4 + 2 * M, oAA = 4 + 2 * M + 2 * M * M;
  for (int w = 0; w < kMwWarps; ++w) {
    if (warp == w) {
#pragma unroll
      for (int r = 0; r < kMwSpl; ++r) {
        const int s = r * 32 + lane;
        if (s < nent && tb) {  // one complex slot per operator
          row[2 * s] += acc_r[r];
          row[2 * s + 1] += acc_i[r];
        } else if (s < nent) {
          const MwEntry e = mw_entry(e_begin + s, M);
          if (e.kind == kEntA) {
            row[oA + 2 * e.i] += acc_r[r];
            row[oA + 2 * e.i + 1] += acc_i[r];
          } else if (e.kind == kEntAdA) {  // <a_j^dag a_i> = conj <a_i^dag a_j>
            row[oM + 2 * (e.i * M + e.j)] += acc_r[r];
            row[oM + 2 * (e.i * M + e.j) + 1] += acc_i[r];
            row[oM + 2 * (e.j * M + e.i)] += acc_r[r];
            row[oM + 2 * (e.j * M + e.i) + 1] -= acc_i[r];
          } else {
            row[oAA + 2 * (e.i * M + e.j)] += acc_r[r];
            row[oAA + 2 * (e.i * M + e.j) + 1] += acc_i[r];
          }
        }
      }
    }
    __syncthreads();
  }
  for (int k = tid; k < nmom; k += kMwBlock) partial[(size_t)blockIdx.x * nmom + k] = row[k];
}

// ------------------------------------------------------------------ host side

template <int MT>
static int launch_prep(const Space& s, const double2* psi, float4* f, double* part, int* grid_out, cudaStream_t st) {
  auto k = obs_prep_kernel<MT>;
  int grid = 0;
  int rc = persistent_grid(k, 0, s.t.total, &grid, kObsBlock);
  if (rc) return rc;
  grid = (int)std::min<int64_t>(grid, max_grid_of(s));
  k<<<grid, kObsBlock, 0, st>>>(s.t, psi, f, part);
  QB_CUDA(cudaGetLastError());
  *grid_out = grid;
  return QB_OK;
}

template <int MT, bool EXACT, int SPL>
static int launch_mw(const Space& s, const double2* psi, const float4* f, double* part, int nmom, int e_begin,
                     int nent, int* grid_out, cudaStream_t st, const float4* ketf, const int* tb) {
  const Tables& t = s.t;
  const int np = (nent + 31) & ~31;
  const int sec_smem = mw_sec_bytes(t) <= kMwSecSmemMax ? 1 : 0;
  constexpr int kMwWarps = mw_warps(SPL), kMwBlock = 32 * kMwWarps;
  const size_t smem = (size_t)(EXACT ? 0 : mw_table_bytes(t)) +
                      mw_smem_after(np, t.nmax, nmom, MwWords<MT, EXACT>::n, MwOccWords<MT>::n, kMwWarps) +
                      (sec_smem ? mw_sec_bytes(t) : 0);
  auto k = moments_w_kernel<MT, EXACT, SPL>;
  int grid = 0;
  int rc = persistent_grid(k, smem, (t.total + 31) / 32 * kMwBlock / kMwWarps, &grid, kMwBlock);
  if (rc) return rc;
  grid = (int)std::min<int64_t>(grid, max_grid_of(s));
  k<<<grid, kMwBlock, smem, st>>>(t, psi, f, part, nmom, e_begin, nent, sec_smem, reinterpret_cast<int*>(s.d_scratch),
                                  ketf, tb);
  QB_CUDA(cudaGetLastError());
  *grid_out = grid;
  return QB_OK;
}

// entries per lane a pass of at most 32 kMwSplMax entries needs, for the mode counts
// with a specialised kernel (M = 5: 30 entries; 7: 56; 9: 90; 11: 132 in passes of
// 96 and 36); the generic kernel takes any
template <int MT, int SPL>
constexpr bool mw_needed() {
  return MT == 0 || (MT == 5 && SPL == 1) || (MT == 7 && SPL == 2) || (MT == 9 && SPL == 3) ||
         (MT == 11 && (SPL == 3 || SPL == 2));
}

template <int MT, bool EXACT>
static int launch_mw_m(const Space& s, const double2* psi, const float4* f, double* part, int nmom, int e_begin,
                       int nent, int* grid, cudaStream_t st, const float4* ketf, const int* tb) {
  // the compiled variant with the fewest entries per lane that holds the pass
  const int spl = (nent + 31) / 32;
  if constexpr (mw_needed<MT, 1>())
    if (spl <= 1) return launch_mw<MT, EXACT, 1>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
  if constexpr (mw_needed<MT, 2>())
    if (spl <= 2) return launch_mw<MT, EXACT, 2>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
  if constexpr (mw_needed<MT, 3>())
    if (spl <= 3) return launch_mw<MT, EXACT, 3>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
  return fail(QB_EINTERNAL, "moments pass without a compiled kernel");
}

// entries per pass of the two-body sweep for M: a multiple of 32 the compiled
// variants take in full passes
static int tb_pass_entries(int M) {
  switch (M) {
    case 5: return 32;
    case 7: return 64;
    case 9: return 96;
    case 11: return 96;
    default: return 32 * kMwSplMax;
  }
}

template <bool EXACT>
static int launch_mw_e(const Space& s, const double2* psi, const float4* f, double* part, int nmom, int e_begin,
                       int nent, int* grid, cudaStream_t st, const float4* ketf = nullptr,
                       const int* tb = nullptr) {
  switch (s.M) {
    case 5: return launch_mw_m<5, EXACT>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
    case 7: return launch_mw_m<7, EXACT>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
    case 9: return launch_mw_m<9, EXACT>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
    case 11: return launch_mw_m<11, EXACT>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
    default: return launch_mw_m<0, EXACT>(s, psi, f, part, nmom, e_begin, nent, grid, st, ketf, tb);
  }
}

// acc[c] += weight * sum_k partial[k][c], in a fixed order
__global__ void accumulate_rows_kernel(const double* partial, int n, int width, double weight, double* acc) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < width; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partial[(size_t)k * width + c];
    acc[c] += weight * s;
  }
}

int launch_tb_bilinear(Space& s, const float4* bra, const float4* ket, const int* d_tb, int n_tb, double weight,
                       double* d_acc, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  // (a pass's partial rows, 2 doubles an entry, live in the moments' partial area)
  const int per = std::min(tb_pass_entries(s.M), std::max(1, nmoments(s.M) / 2));
  for (int e0 = 0; e0 < n_tb; e0 += per) {
    const int ne = std::min(per, n_tb - e0);
    int gm = 0;
    int rc = s.t.exact ? launch_mw_e<true>(s, nullptr, bra, partial_area(s), 2 * ne, e0, ne, &gm, st, ket, d_tb)
                       : launch_mw_e<false>(s, nullptr, bra, partial_area(s), 2 * ne, e0, ne, &gm, st, ket, d_tb);
    if (rc) return rc;
    accumulate_rows_kernel<<<(2 * ne + 127) / 128, 128, 0, st>>>(partial_area(s), gm, 2 * ne, weight, d_acc + 2 * e0);
    QB_CUDA(cudaGetLastError());
  }
  return QB_OK;
}

int launch_moments(Space& s, const void* d_psi, double* out_host, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int M = s.M, nmom = nmoments(M), npr = nprep(M);
  const double2* psi = (const double2*)d_psi;
  float4* f = s.d_obsf;
  // pass 1: weighted copy, norm, <N>, <n_i>
  int gp = 0;
  int rc;
  switch (M) {
    case 5: rc = launch_prep<5>(s, psi, f, prep_area(s), &gp, st); break;
    case 7: rc = launch_prep<7>(s, psi, f, prep_area(s), &gp, st); break;
    case 9: rc = launch_prep<9>(s, psi, f, prep_area(s), &gp, st); break;
    case 11: rc = launch_prep<11>(s, psi, f, prep_area(s), &gp, st); break;
    default: rc = launch_prep<0>(s, psi, f, prep_area(s), &gp, st); break;
  }
  if (rc) return rc;
  reduce_rows_kernel<<<1, 32, 0, st>>>(prep_area(s), gp, npr, prep_final(s));
  QB_CUDA(cudaGetLastError());
  // pass 3: <psi|H|psi> from the weighted copy, w^2 applied per row in FP64
  DfArgs a{};
  a.vin = f;
  a.diag = s.d_diag;
  a.scale[0] = make_float2(1.0f, 0.0f);
  a.row0 = 0;
  a.row1 = s.t.total;
  a.status = reinterpret_cast<int*>(s.d_scratch);
  a.partial = dot_area(s);
  int g2 = 0;
  rc = stage_launch(s.t, a, 4, 1, s.t.is_complex != 0, st, &g2, false, 0);
  if (rc) return rc;
  reduce_rows_kernel<<<1, 32, 0, st>>>(a.partial, g2, 1, dot_final(s));
  QB_CUDA(cudaGetLastError());
  // pass 2: the moments that move the ket, in passes of at most 32 kMwSplMax entries;
  // each pass's partial rows are summed into its own copy of the moment row
  const int nent = mw_entries(M), per = 32 * kMwSplMax;
  const int npass = (nent + per - 1) / per;
  std::vector<double> mom((size_t)nmom, 0.0), fin((size_t)nmom);
  for (int p = 0; p < npass; ++p) {
    const int e0 = p * per, ne = std::min(per, nent - e0);
    int gm = 0;
    rc = s.t.exact ? launch_mw_e<true>(s, psi, f, partial_area(s), nmom, e0, ne, &gm, st)
                   : launch_mw_e<false>(s, psi, f, partial_area(s), nmom, e0, ne, &gm, st);
    if (rc) return rc;
    reduce_rows_kernel<<<(nmom + 127) / 128, 128, 0, st>>>(partial_area(s), gm, nmom, final_area(s));
    QB_CUDA(cudaGetLastError());
    QB_CUDA(cudaMemcpyAsync(fin.data(), final_area(s), sizeof(double) * nmom, cudaMemcpyDeviceToHost, st));
    QB_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < nmom; ++k) mom[k] += fin[k];
  }
  std::vector<double> pre((size_t)npr);
  double h = 0.0;
  QB_CUDA(cudaMemcpyAsync(pre.data(), prep_final(s), sizeof(double) * npr, cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaMemcpyAsync(&h, dot_final(s), sizeof(double), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < nmom; ++k) out_host[k] = mom[k];
  out_host[0] = pre[0];
  out_host[1] = pre[1];
  out_host[2] = h;
  out_host[3] = 0.0;
  const int oM = 4 + 2 * M;
  for (int i = 0; i < M; ++i) {
    out_host[oM + 2 * (i * M + i)] = pre[2 + i];
    out_host[oM + 2 * (i * M + i) + 1] = 0.0;
  }
  return check_status(s, st);
}

}  // namespace qb
