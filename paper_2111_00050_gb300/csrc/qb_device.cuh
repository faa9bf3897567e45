// Device-side building blocks shared by the qb kernels: the shared-memory view
// of a space's tables, row unranking into suffix states, double-float
// arithmetic and the persistent-grid helper.  Internal; see qb_internal.h.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "qb_internal.h"

namespace qb {

#define QB_CUDA(x)                                                                            \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return fail(QB_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kBlock = 128;  // threads per CTA of the row kernels (one row per thread per pass)
constexpr int kMaxM = QB_MAX_MODES;

// ----------------------------------------------------------------- smem view

struct View {
  const uint32_t* cnt;
  const int32_t* E;
  const double* sq;
  const uint32_t* pq;
  const double* G;
  const int8_t* delta;
  const int32_t* ann;
  const int32_t* hs;
  const uint8_t* pairidx;
  const double* w;
  const double* gd;
};

// Table pointers for an image whose byte 0 is at s (pointer arithmetic only).
__device__ __forceinline__ View view_at(const Tables& t, const unsigned char* s) {
  View v;
  v.cnt = (const uint32_t*)(s + t.o_cnt);
  v.E = (const int32_t*)(s + t.o_E);
  v.sq = (const double*)(s + t.o_sqrt);
  v.pq = (const uint32_t*)(s + t.o_pq);
  v.G = (const double*)(s + t.o_G);
  v.delta = (const int8_t*)(s + t.o_delta);
  v.ann = (const int32_t*)(s + t.o_ann);
  v.hs = (const int32_t*)(s + t.o_hs);
  v.pairidx = (const uint8_t*)(s + t.o_pairidx);
  v.w = (const double*)(s + t.o_w);
  v.gd = (const double*)(s + t.o_gd);
  return v;
}

// Bytes of the table image a row kernel stages in shared memory: everything from
// t.sm_from on (the fill counts and the ranking table stay in global memory for
// exact momentum, where they are large).
__host__ __device__ inline size_t blob_smem(const Tables& t) {
  return ((size_t)(t.blob_bytes - t.sm_from) + 15) & ~(size_t)15;
}

// Copies the row kernels' part of the table image into shared memory (16-byte
// vector copies).
__device__ __forceinline__ void load_blob(const Tables& t, unsigned char* smem) {
  const int4* src = reinterpret_cast<const int4*>(t.blob + t.sm_from);
  int4* dst = reinterpret_cast<int4*>(smem);
  for (int i = threadIdx.x; i < (t.blob_bytes - t.sm_from) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// Table pointers of a row kernel after load_blob: the staged tables in shared
// memory, the ones below t.sm_from in global memory.
__device__ __forceinline__ View make_view(const Tables& t, const unsigned char* staged) {
  View v = view_at(t, staged - t.sm_from);
  if (t.o_cnt < t.sm_from) v.cnt = reinterpret_cast<const uint32_t*>(t.blob + t.o_cnt);
  if (t.o_E < t.sm_from) v.E = reinterpret_cast<const int32_t*>(t.blob + t.o_E);
  return v;
}

// Flat-index shift of term j's target suffix state at mode m (biased bytes, or
// plain int16 for exact momentum).
__device__ __forceinline__ int delta_shift(const Tables& t, const View& v, int j, int m) {
  if (t.exact) return (int)reinterpret_cast<const int16_t*>(v.delta)[j * 16 + m];
  return (int)reinterpret_cast<const uint8_t*>(v.delta)[j * 16 + m] - kDeltaBias;
}

// Copies the table image from byte offset `from` on (16-byte aligned) into
// shared memory; the stage kernels leave the fill counts in global memory.
__device__ __forceinline__ void load_blob_from(const Tables& t, unsigned char* smem, int from) {
  const int4* src = reinterpret_cast<const int4*>(t.blob + from);
  int4* dst = reinterpret_cast<int4*>(smem);
  for (int i = threadIdx.x; i < (t.blob_bytes - from) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// Per-thread scratch rows in shared memory, laid out [m][thread] so that the
// lanes of a warp touching the same mode hit consecutive words.
struct RowScratch {
  uint8_t* occ;  // [kMaxM][kBlock]
  int32_t* idx;  // [kMaxM][kBlock] flat E index of the suffix state at mode m
  int32_t* pe;   // [kMaxM][kBlock] prefix sums of E over the row's own suffix states
};

__device__ __forceinline__ RowScratch row_scratch(unsigned char* base) {
  RowScratch r;
  r.idx = reinterpret_cast<int32_t*>(base);
  r.pe = r.idx + kMaxM * kBlock;
  r.occ = reinterpret_cast<uint8_t*>(r.pe + kMaxM * kBlock);
  return r;
}
constexpr int kRowScratchBytes = kMaxM * kBlock * (4 + 4 + 1);

__device__ __forceinline__ int find_sector(const Tables& t, int64_t g) {
  int lo = 0, hi = t.n_sectors - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(t.sec_off + mid) <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Unranks local index i of sector (N, K) into the occupation vector and fills
// the suffix-state indices and their prefix sums.  Returns rank(n) recomputed
// from the suffix states (equals i for a consistent table).
__device__ __forceinline__ int64_t setup_row(const Tables& t, const View& v, const RowScratch& rs, int N, int K,
                                             int64_t D, int64_t i) {
  const int M = t.M, Q = t.Q, tid = threadIdx.x, V = t.nmax + 1;
  int rem = N, kr = K;
  int64_t left = i;
  for (int m = 0; m < M - 1; ++m) {
    int val = 0, kk = kr;
    const uint32_t* row = v.cnt + (size_t)(m + 1) * V * Q;
    while (true) {
      uint32_t c = row[(rem - val) * Q + kk];
      if (left < (int64_t)c || val == rem) break;
      left -= c;
      ++val;
      kk -= m;
      if (kk < 0) kk += Q;
    }
    rs.occ[m * kBlock + tid] = (uint8_t)val;
    rem -= val;
    kr = kk;
  }
  rs.occ[(M - 1) * kBlock + tid] = (uint8_t)rem;
  // suffix states, from the top mode down
  const int twoQ = 2 * Q;
  int srem = 0, skr = 0;
  for (int m = M - 1; m >= 1; --m) {
    int nm = rs.occ[m * kBlock + tid];
    srem += nm;
    skr = (skr + m * nm) % Q;
    rs.idx[m * kBlock + tid] = (m * t.rem_w + srem + 2) * twoQ + skr;
  }
  int32_t acc = 0;
  rs.pe[tid] = 0;
  for (int m = 1; m < M; ++m) {
    acc += v.E[rs.idx[m * kBlock + tid]];
    rs.pe[m * kBlock + tid] = acc;
  }
  return D - 1 - (int64_t)acc;
}

// Ket weight w(n) = sqrt(N! / prod_m n_m!) 2^-e_N and its inverse in FP64, from the
// occupations occ[m * stride]: the product over modes of sqrt(C(rem_m, n_m)), times the
// power of two that centres the weights of N particles on 1 (Tables::wscale).  In the
// weighted basis f = psi / w the two-body matrix element of a pair (r, s) -> (p, q)
// loses its creation factor sqrt((n_p + 1)(n_q + 1 + [p = q])) (see the stage kernel).
template <int MT>
__device__ __forceinline__ double2 ket_weight(const Tables& t, const uint8_t* occ, int stride) {
  const int M = (MT > 0) ? MT : t.M;
  constexpr int kMB = (MT > 0) ? MT : 16;
  int rem = 0;
#pragma unroll
  for (int m = 0; m < kMB; ++m)
    if (m < M) rem += occ[m * stride];
  const int V = t.nmax + 1;
  const double2 c = __ldg(t.wscale + rem);  // rem = N here
  double w = 1.0, wi = 1.0;
#pragma unroll
  for (int m = 0; m < kMB - 1; ++m) {
    if (m >= M - 1) break;
    const int nm = occ[m * stride];
    const double2 f = __ldg(t.wtab + rem * V + nm);
    w *= f.x;
    wi *= f.y;
    rem -= nm;
  }
  return make_double2(w * c.x, wi * c.y);
}

// n_m of a packed occupation word (Tables::occ)
__device__ __forceinline__ int occ_of(uint64_t word, int m, int ob) {
  return (int)((uint32_t)(word >> (m * ob)) & ((1u << ob) - 1u));
}

// ket_weight from a packed occupation word: the same products in the same order
template <int MT>
__device__ __forceinline__ double2 ket_weight_word(const Tables& t, uint64_t word) {
  const int M = (MT > 0) ? MT : t.M;
  constexpr int kMB = (MT > 0) ? MT : 16;
  const int ob = t.occ_bits;
  int rem = 0;
#pragma unroll
  for (int m = 0; m < kMB; ++m)
    if (m < M) rem += occ_of(word, m, ob);
  const int V = t.nmax + 1;
  const double2 c = __ldg(t.wscale + rem);
  double w = 1.0, wi = 1.0;
#pragma unroll
  for (int m = 0; m < kMB - 1; ++m) {
    if (m >= M - 1) break;
    const int nm = occ_of(word, m, ob);
    const double2 f = __ldg(t.wtab + rem * V + nm);
    w *= f.x;
    wi *= f.y;
    rem -= nm;
  }
  return make_double2(w * c.x, wi * c.y);
}

// Rank of the ket obtained from the row's ket by changing the occupations of
// modes e[0..nch) by dn[0..nch), inside the sector of dimension Dt it lands in.
__device__ __forceinline__ int64_t rank_changed(const Tables& t, const View& v, const RowScratch& rs, int nch,
                                                const int* e, const int* dn, int64_t Dt) {
  const int M = t.M, Q = t.Q, tid = threadIdx.x, twoQ = 2 * Q;
  int top = 0;
  for (int c = 0; c < nch; ++c) top = max(top, e[c]);
  if (top > M - 1) top = M - 1;
  int64_t sum = rs.pe[(M - 1) * kBlock + tid] - rs.pe[top * kBlock + tid];
  int dc = 0, dk = 0;
  for (int m = top; m >= 1; --m) {
    for (int c = 0; c < nch; ++c)
      if (e[c] == m) {
        dc += dn[c];
        dk += dn[c] * m;
      }
    int dkm = ((dk % Q) + Q) % Q;
    sum += v.E[rs.idx[m * kBlock + tid] + dc * twoQ + dkm];
  }
  return Dt - 1 - sum;
}

// ------------------------------------------------ double-float RK4 stages
//
// GB300's FP64 pipe runs at about 1/74 of the FP32 rate, so the gather-heavy
// stages accumulate in double-float arithmetic: a value is the unevaluated sum
// hi + lo of two fp32 numbers (about 48 significant bits).  Products use the
// exact fma-based error term, sums the branch-free TwoSum; the intrinsics
// __fmul_rn / __fadd_rn keep the compiler from contracting them.  The state
// psi itself stays FP64: the last stage of each step forms psi + z H v in FP64.

struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// a * k for a float k that is an exact small integer, unnormalised
__device__ __forceinline__ dfl df_mul_f(dfl a, float k) {
  const float p = __fmul_rn(a.h, k);
  float e = fmaf(a.h, k, -p);
  e = fmaf(a.l, k, e);
  return {p, e};
}

// a * b, unnormalised (|l| is a few ulp of h)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return {p, e};
}

// acc += c * x; acc.h carries the TwoSum, acc.l gathers every rounding error
__device__ __forceinline__ void df_fma(dfl& acc, dfl c, dfl x) {
  const float p = __fmul_rn(c.h, x.h);
  float e = fmaf(c.h, x.h, -p);
  e = fmaf(c.h, x.l, e);
  e = fmaf(c.l, x.h, e);
  const float s = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

// a + b, renormalised
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  err = __fadd_rn(err, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, err);
  return {h, __fsub_rn(err, __fsub_rn(h, s))};
}

// Fast two-sum renormalisation of a pair whose |l| may have grown to a few ulp of h
__device__ __forceinline__ dfl df_renorm(dfl a) {
  const float h = __fadd_rn(a.h, a.l);
  return {h, __fsub_rn(a.l, __fsub_rn(h, a.h))};
}

// A double-float complex value is stored as float4 (re.hi, im.hi, re.lo, im.lo),
// so that a load yields the packed pairs (re.hi, im.hi) and (re.lo, im.lo).
__device__ __forceinline__ float4 df_pack(dfl re, dfl im) { return make_float4(re.h, im.h, re.l, im.l); }
__device__ __forceinline__ dfl df_re(float4 v) { return {v.x, v.z}; }
__device__ __forceinline__ dfl df_im(float4 v) { return {v.y, v.w}; }

// Packed pairs of fp32 (lane 0 in the low word) and the correctly rounded
// two-lane arithmetic of sm_100+ (add/sub/mul/fma .rn.f32x2).
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Two double-float numbers side by side: hi words (lane0, lane1), lo words likewise.
struct dfc {
  f2 h, l;
};

// acc += c * x lane by lane, with per-lane double-float coefficient c = (ch, cl)
// (nch = -ch) and double-float x = (xh, xl): the fma-based exact product error and
// TwoSum of the scalar df_fma, two lanes per instruction.
__device__ __forceinline__ void dfc_fma(dfc& acc, f2 ch, f2 nch, f2 cl, f2 xh, f2 xl) {
  const f2 pn = f2_mul(nch, xh);  // -fl(c.h x.h)
  f2 e = f2_fma(ch, xh, pn);      // exact error of that product
  e = f2_fma(ch, xl, e);
  e = f2_fma(cl, xh, e);
  const f2 s = f2_sub(acc.h, pn);  // acc.h + p
  const f2 bb = f2_sub(s, acc.h);
  const f2 err = f2_sub(f2_sub(acc.h, f2_sub(s, bb)), f2_add(pn, bb));  // (a - (s - bb)) + (p - bb)
  acc.h = s;
  acc.l = f2_add(acc.l, f2_add(err, e));
}

__device__ __forceinline__ dfc dfc_renorm(dfc a) {
  const f2 h = f2_add(a.h, a.l);
  return {h, f2_sub(a.l, f2_sub(h, a.h))};
}

// Arguments of one stage launch.  With z = -i zre and x the gathered vector
// (vin), the epilogue writes, by `mode`:
//   0  out  = psif + z H x                        (forward Horner stage, d > 1)
//   1  psi += z H x;          out = df(psi)       (forward final stage, FP64 psi)
//   2  out  = z H x                               (adjoint: costate stage vector)
//   3  psi += sum_k basef[k] + z H x; out = df(psi)  (adjoint: new costate, FP64)
//   4  no output; with bilinears on, partial[block][0] = sum Re(conj(x_i) (H x)_i)
// For the adjoint pass zre = -c dt, i.e. z = +i c dt.  With bilinears on, every
// row also adds Im <pair_i, H_L x_i> and n_q(i) Im(conj(x_i) pair_i) to per-CTA
// sums written to partial[block][M + 1] (H_L: the two-body part at scale 1).
struct DfArgs {
  const float4* vin;   // gathered stage vector(s), double-float [B][total]
  const float4* psif;  // double-float copy of psi [B][total] (mode 0)
  double2* psi;        // FP64 vector updated in place (modes 1, 3)
  float4* out;         // double-float output [B][total]
  const float4* basef[3];  // mode 3: double-float vectors added to psi
  int nbasef;
  const float4* pair;  // bilinear pair vector (double-float), own row only
  double* partial;     // bilinear sums [gridDim.x][M + 1]
  const float4* diag;  // per ket (w.hi, w.lo, L.hi, L.lo)
  float2 scale[8];     // two-body scale per member, double-float
  int64_t row0, row1;  // kets [row0, row1) of the launch (every sector: 0, total)
  double zre;          // z = -i zre
  float2 zf;           // zre as double-float
  int* status;
};

// Resident CTAs per SM of `kernel` with `smem` dynamic shared memory, cached
// per (kernel, smem) so that launch loops do not repeat the occupancy query.
template <typename K>
static int occupancy_cached(K kernel, size_t smem, int* per_sm, int* sms, int block = kBlock) {
  struct Entry {
    const void* fn;
    size_t smem;
    int dev, per, sms;
  };
  static thread_local Entry cache[64];
  static thread_local int used = 0;
  int dev = 0;
  QB_CUDA(cudaGetDevice(&dev));
  const void* fn = reinterpret_cast<const void*>(kernel);
  for (int i = 0; i < used; ++i)
    if (cache[i].fn == fn && cache[i].smem == smem && cache[i].dev == dev) {
      *per_sm = cache[i].per;
      *sms = cache[i].sms;
      return QB_OK;
    }
  int s = 0, per = 0, optin = 0;
  QB_CUDA(cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev));
  // The dynamic shared-memory limit is a property of the function shared by every
  // space: raise it once to the device maximum so that no later call lowers it.
  QB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  QB_CUDA(cudaFuncGetAttributes(&fa, kernel));
  if (smem + fa.sharedSizeBytes > (size_t)optin)
    return fail(QB_EUNSUPPORTED, "tables too large for shared memory (reduce n_max or M)");
  QB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes));
  QB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, smem));
  if (per < 1) return fail(QB_EUNSUPPORTED, "kernel does not fit on an SM with this table size");
  Entry e{fn, smem, dev, per, s};
  cache[used < 64 ? used++ : 63] = e;
  *per_sm = per;
  *sms = s;
  return QB_OK;
}

// Persistent grid of a row kernel: at most one wave of resident CTAs (capped at
// 16 per SM, the size the reduction scratch is planned for), no more CTAs than
// there are block-row tiles.
template <typename K>
static int persistent_grid(K kernel, size_t smem, int64_t rows, int* grid, int block = kBlock) {
  int per = 0, sms = 0;
  int rc = occupancy_cached(kernel, smem, &per, &sms, block);
  if (rc) return rc;
  int64_t want = (rows + block - 1) / block;
  int64_t g = std::min<int64_t>((int64_t)sms * std::min(per, 16), std::max<int64_t>(1, want));
  *grid = (int)g;
  return QB_OK;
}

}  // namespace qb
