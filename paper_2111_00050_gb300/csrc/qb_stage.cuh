// The hot kernel: one Horner RK4 stage of every sector (and every member of a
// batched coupling sweep) in one launch, with the matrix-free sector H psi in
// double-float arithmetic.
//
//   stage d (d = 4, 3, 2):  out = psi + (-i dt/d) H v     (double-float out)
//   stage 1:                psi = psi + (-i dt) H v       (FP64 psi, plus its
//                                                          double-float copy)
//
// H is Eq. (Ham) restricted to sectors of fixed N and momentum mod M
// (Sec. III B).  Per row (ket n) the off-diagonal terms are the disjoint pairs
// {r, s} -> {p, q} with p + q = r + s (mod M): coefficient
// G_{pq,rs} sqrt(n_r (n_s - [r=s])) sqrt((n_p + 1)(n_q + 1 + [p=q])), G the
// multiplicity-summed symmetrised coupling; the diagonal is precomputed per ket.
//
// Work layout: every warp owns tiles of kWarpRows consecutive kets and runs
// without CTA-wide barriers.  Phase 1 unranks the tile (kWarpRows/32 kets per
// lane) into occupations and suffix-state indices; phase 2 counting-sorts the
// tile by the number of annihilation pairs acting on each ket; phase 3 runs the
// terms in rounds, the 32 lanes of a round taking 32 kets of nearly equal work.
// For odd M every annihilation pair has exactly (M-1)/2 creation partners; the
// specialised kernels unroll them so that their ranks and gathers overlap.
#pragma once
#include "qb_device.cuh"

#ifndef QB_CNT_GLOBAL
#define QB_CNT_GLOBAL 1
#endif
#ifndef QB_UNROLL_PARTNERS
#define QB_UNROLL_PARTNERS 1
#endif
#ifndef QB_CONVERGENT_PAIRS
#define QB_CONVERGENT_PAIRS 1
#endif
#ifndef QB_UNRANK_FROM_E
#define QB_UNRANK_FROM_E 1
#endif
// 1: a ket's occupations are unpacked from the packed table Tables::occ (8 B per ket
// read, coalesced); 0: unranked through the counting table (a data-dependent walk of
// about N + M steps per ket)
#ifndef QB_OCC_TABLE
#define QB_OCC_TABLE 1
#endif

namespace qb {

// Warps per CTA of the stage kernel.  The CTA's warps share one copy of the
// ranking table in shared memory, so larger CTAs leave room for more warps per SM.
#ifndef QB_STAGE_WARPS
#define QB_STAGE_WARPS 12
#endif
// Resident CTAs per SM that the register budget of the single-state stage kernel
// is planned for: 3 x 384 threads leave 56 registers per thread (36 warps per SM).
// The bilinear instantiations (more accumulators per lane) of the specialised mode
// counts are planned for 2 CTAs (80 registers); the batched ones and the generic
// bilinear ones (16 accumulators) keep the compiler's choice (one CTA).
#ifndef QB_STAGE_MIN_BLOCKS
#define QB_STAGE_MIN_BLOCKS 3
#endif
constexpr int kStageWarps = QB_STAGE_WARPS;
constexpr int kStageBlock = 32 * kStageWarps;
constexpr int kStageMinBlocks = QB_STAGE_MIN_BLOCKS;

// first byte of the table image the stage kernels stage in shared memory
// (exact momentum: the ranking table too stays in global memory)
__host__ __device__ inline int kSmemFrom(const Tables& t, bool exact = false) {
  return exact ? t.o_sqrt : (QB_CNT_GLOBAL ? t.o_E : 0);
}

// Gathered stage-vector entry: read-only global load, or a generic load when the
// vector is a shared-memory copy (LOCAL; the non-coherent global path does not
// accept shared addresses).
template <bool LOCAL>
__device__ __forceinline__ float4 gather(const float4* p) {
  if (LOCAL) return *p;
  return __ldg(p);
}

// E at suffix index id shifted by `shift` entries.  BYTE: id is a byte offset, so a
// lookup is one shift-add onto it (measured: 6% faster where the ranking table is
// in global memory, exact momentum; 2% slower from shared memory).
template <bool BYTE>
__device__ __forceinline__ int32_t e_at(const int32_t* E, int id, int shift) {
  if (BYTE) return *reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(E) + id + (shift << 2));
  return E[id + shift];
}

// One warp tile: kets [base, min(base + kWarpRows, row1)) of the launch.  With
// LOCAL the state vectors of DfArgs are the shared-memory copies of one sector
// starting at ket local_off (gathers and own-row accesses are sector-local);
// otherwise they are the global vectors.  The per-ket diagonal is always global.
//
// SIM: the double-float vectors hold f = psi / w in the weighted basis of the ket
// weights w(n) = sqrt(N! / prod n_m!) (modes 0 to 3).  The similar matrix
// W^-1 H W has the same diagonal, and for the target n' = n - e_r - e_s + e_p + e_q
// of a term, w(n') / w(n) = sqrt(n_r (n_s - [r = s]) / ((n_p + 1)(n_q + 1 + [p = q]))),
// so its element is G n_r (n_s - [r = s]): an integer times the coupling, with no
// creation-side square roots and no lookup of n_p, n_q.  Modes 1 and 3 map back:
// psi += w (z W^-1 H W f + sum of basef) in FP64, and write f = psi_new / w; the
// bilinears multiply each factor by w.
//
// EXACT: momentum conserved exactly: momentum arithmetic modulo t.Q > every
// momentum sum, shifts stored as int16, the ranking table in global memory.
template <int MT, int B, bool CPLX, bool BIL, bool LOCAL, bool SIM, bool EXACT>
__device__ __forceinline__ void stage_tile(const Tables& t, const View& v, const float2* sqf, const float4* Gf,
                                           const uint4* dl4, const DfArgs& a, const int mode, const int64_t base,
                                           const int64_t row1, const int64_t local_off, int32_t* sidx, uint8_t* socc,
                                           int32_t* sD, int64_t* sOff, uint8_t* sperm, int32_t* hist,
                                           int32_t* cursor, dfl& bil_l, dfl* bil_w) {
  const int M = (MT > 0) ? MT : t.M;
  const int Qm = EXACT ? t.Q : M;  // momentum modulus
  const int twoM = 2 * Qm;         // row width of the ranking table
  const int lane = threadIdx.x & 31;
  const int64_t total = t.total;  // stride between sweep members
  const int nb = t.n_ann + 2;
  constexpr int kMB = (MT > 0) ? MT : 16;
  // ---- phase 1: each lane unpacks (or unranks) kWarpRows/32 kets into occupations and suffix-state indices
  for (int k = lane; k < 2 * nb; k += 32) hist[k] = 0;
  int key[kWarpRows / 32];
#pragma unroll
  for (int u = 0; u < kWarpRows / 32; ++u) {
    const int row = u * 32 + lane;
    const int64_t g = base + row;
    key[u] = 0;
    if (g < row1) {
      const int sid = find_sector(t, g);
      const int64_t off = __ldg(t.sec_off + sid);
      const int D = (int)(__ldg(t.sec_off + sid + 1) - off);
#if QB_OCC_TABLE
      {
        const uint64_t word = __ldg(t.occ + g);
        const int ob = t.occ_bits;
        const uint32_t omask = (1u << ob) - 1u;
        for (int m = 0; m < M; ++m) socc[m * kWarpRows + row] = (uint8_t)((uint32_t)(word >> (m * ob)) & omask);
      }
#else
      int rem = __ldg(t.sec_N + sid), kr = __ldg(t.sec_K + sid);
      int left = (int)(g - off);
      for (int m = 0; m < M - 1; ++m) {
        int val = 0, kk = kr;
#if QB_UNRANK_FROM_E
        // cnt[m+1][n][k] = E_{m+2}(n + 1, k + m + 1), already in shared memory; for
        // the last step cnt[M-1][n][k] = [n + k = 0 mod M] (one mode left)
        const int32_t* erow = v.E + (min(m + 2, M - 1) * t.rem_w + 3) * twoM + m + 1;  // used for m + 2 < M
        while (true) {
          const int c = (m + 2 < M)  ? erow[(rem - val) * twoM + kk]
                        : EXACT      ? ((M - 1) * (rem - val) == kk ? 1 : 0)
                                     : (((rem - val + kk) % M) == 0 ? 1 : 0);
#else
        const uint32_t* crow = gcnt + (size_t)(m + 1) * V * M;
        while (true) {
          const int c = (int)crow[(rem - val) * M + kk];
#endif
          if (left < c || val == rem) break;
          left -= c;
          ++val;
          kk -= m;
          if (kk < 0) kk += Qm;
        }
        socc[m * kWarpRows + row] = (uint8_t)val;
        rem -= val;
        kr = kk;
      }
      socc[(M - 1) * kWarpRows + row] = (uint8_t)rem;
#endif
      int srem = 0, skr = 0, esum = 0, np = 0, n2 = 0;
      for (int m = M - 1; m >= 1; --m) {
        const int nm = socc[m * kWarpRows + row];
        srem += nm;
        skr += m * nm;
        while (skr >= Qm) skr -= Qm;
        const int ix = (m * t.rem_w + srem + 2) * twoM + skr;
        esum += v.E[ix];
        sidx[m * kWarpRows + row] = EXACT ? ix * 4 : ix - kDeltaBias;
      }
      if (D - 1 - esum != (int)(g - off)) atomicOr(a.status, 2);
      for (int m = 0; m < M; ++m) {
        const int nm = socc[m * kWarpRows + row];
        np += nm >= 1;
        n2 += nm >= 2;
      }
      key[u] = np * (np - 1) / 2 + n2;  // annihilation pairs r <= s acting on the ket
      sD[row] = D;
      sOff[row] = off;
    } else {
      sD[row] = -1;
    }
  }
  // ---- phase 2: warp-local counting sort of the tile by work, largest first
  __syncwarp();
#pragma unroll
  for (int u = 0; u < kWarpRows / 32; ++u) atomicAdd(&hist[key[u]], 1);
  __syncwarp();
  if (lane == 0) {
    int run = 0;
    for (int k = nb - 1; k >= 0; --k) {
      cursor[k] = run;
      run += hist[k];
    }
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < kWarpRows / 32; ++u) sperm[atomicAdd(&cursor[key[u]], 1)] = (uint8_t)(u * 32 + lane);
  __syncwarp();

  // ---- phase 3: rounds of 32 kets of similar work, one per lane
  for (int round = 0; round < kWarpRows / 32; ++round) {
    const int row = sperm[round * 32 + lane];
    const int D = sD[row];
    if (D < 0) continue;
    const int64_t off = sOff[row];
    const int64_t gr = base + row;
    const int64_t ri = LOCAL ? gr - local_off : gr;  // own-row index into the state vectors
    const uint8_t* occ = socc + row;
    int id[16];
#pragma unroll
    for (int m = 1; m < 16; ++m)
      if (m < M) id[m] = sidx[m * kWarpRows + row];
    uint32_t occmask = 0, twomask = 0;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (m >= M) break;
      const int nm = occ[m * kWarpRows];
      occmask |= (nm >= 1 ? 1u : 0u) << m;
      twomask |= (nm >= 2 ? 1u : 0u) << m;
    }
    const float4* vsec = a.vin + (LOCAL ? 0 : off);  // gathers
    dfc acc[B];  // (re, im) of the off-diagonal sum, double-float, packed
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = dfc{0ull, 0ull};

#if QB_CONVERGENT_PAIRS
    // One annihilation pair (r <= s, n_r (n_s - [r=s]) > 0) per iteration.  Kets of
    // a round have (nearly) the same pair count, so the iterations line up across
    // the warp; the search for the next r is a short inner loop.
    const int np = __popc(occmask);
    const int npairs = np * (np - 1) / 2 + __popc(twomask);
    uint32_t rm = occmask, smask = 0;
    int r = 0;
    for (int it = 0; it < npairs; ++it) {
      while (smask == 0 && rm != 0) {
        r = __ffs(rm) - 1;
        rm &= rm - 1;
        smask = occmask & (~0u << r);
        if (!((twomask >> r) & 1u)) smask &= ~(1u << r);
      }
      if (smask == 0) break;  // not reached: npairs counts exactly the pairs found here
#else
    uint32_t rm = occmask, smask = 0;
    int r = 0;
    while (true) {
      if (smask == 0) {
        if (rm == 0) break;
        r = __ffs(rm) - 1;
        rm &= rm - 1;
        smask = occmask & (~0u << r);
        if (!((twomask >> r) & 1u)) smask &= ~(1u << r);
        if (smask == 0) continue;
      }
#endif
      const int s = __ffs(smask) - 1;
      smask &= smask - 1;
      const int ai = v.pairidx[r * 16 + s];
      dfl A{0.f, 0.f};  // sqrt(n_r (n_s - [r = s]))
      float Af = 0.f;   // n_r (n_s - [r = s]), exact (SIM)
      if (SIM) {
        Af = (float)(occ[r * kWarpRows] * (occ[s * kWarpRows] - (r == s ? 1 : 0)));
      } else {
        const float2 sa = sqf[occ[r * kWarpRows]], sb = sqf[occ[s * kWarpRows] - (r == s ? 1 : 0)];
        A = df_mul(dfl{sa.x, sa.y}, dfl{sb.x, sb.y});
      }
      // (exact momentum: the partner count varies from pair to pair)
      constexpr int kC = (QB_UNROLL_PARTNERS && !CPLX && !EXACT && MT > 0 && (MT % 2) == 1) ? (MT - 1) / 2 : 0;
      if (kC > 0) {
        // fixed partner count: all ranks first, then all gathers, then the sums
        const int j0 = v.ann[ai];
        int rkc[kC > 0 ? kC : 1];
        dfl crc[kC > 0 ? kC : 1];
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          const int j = j0 + c;
          dfl AB{0.f, 0.f};
          if (!SIM) {
            const uint32_t w4 = v.pq[j];
            const int p = w4 & 0xff, q = (w4 >> 8) & 0xff;
            const float2 bp = sqf[occ[p * kWarpRows] + 1], bq = sqf[occ[q * kWarpRows] + 1 + (p == q ? 1 : 0)];
            AB = df_mul(A, df_mul(dfl{bp.x, bp.y}, dfl{bq.x, bq.y}));
          }
          const uint4 dd = dl4[j];
          int esum = 0;
#pragma unroll
          for (int m = 1; m < 16; ++m) {
            if (m >= M) break;
            const uint32_t word = (m < 4) ? dd.x : (m < 8) ? dd.y : (m < 12) ? dd.z : dd.w;
            esum += e_at<EXACT>(v.E, id[m], (int)((word >> (8 * (m & 3))) & 0xffu));
          }
          int rk = D - 1 - esum;
          if ((unsigned)rk >= (unsigned)D) {
            atomicOr(a.status, 1);
            rk = 0;
          }
          rkc[c] = rk;
          const float4 gf = Gf[j];
          crc[c] = SIM ? df_mul_f(dfl{gf.x, gf.y}, Af) : df_mul(dfl{gf.x, gf.y}, AB);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          float4 x[kC > 0 ? kC : 1];
#pragma unroll
          for (int c = 0; c < kC; ++c) x[c] = gather<LOCAL>(vsec + (size_t)b * total + rkc[c]);
#pragma unroll
          for (int c = 0; c < kC; ++c)
            dfc_fma(acc[b], f2_pack(crc[c].h, crc[c].h), f2_pack(-crc[c].h, -crc[c].h),
                    f2_pack(crc[c].l, crc[c].l), f2_pack(x[c].x, x[c].y), f2_pack(x[c].z, x[c].w));
        }
      } else {
        const int j1 = v.ann[ai + 1];
        for (int j = v.ann[ai]; j < j1; ++j) {
          dfl AB{0.f, 0.f};
          if (!SIM) {
            const uint32_t w4 = v.pq[j];
            const int p = w4 & 0xff, q = (w4 >> 8) & 0xff;
            const float2 bp = sqf[occ[p * kWarpRows] + 1], bq = sqf[occ[q * kWarpRows] + 1 + (p == q ? 1 : 0)];
            AB = df_mul(A, df_mul(dfl{bp.x, bp.y}, dfl{bq.x, bq.y}));
          }
          // rank of the target: D - 1 - sum over every mode of E at the shifted suffix state
          int esum = 0;
          if (EXACT) {  // int16 shifts, two modes per word
            const uint4 d0 = dl4[2 * j], d1 = dl4[2 * j + 1];
  #pragma unroll
            for (int m = 1; m < 16; ++m) {
              if (m >= M) break;
              const uint32_t word = (m < 2) ? d0.x : (m < 4) ? d0.y : (m < 6) ? d0.z : (m < 8) ? d0.w
                                  : (m < 10) ? d1.x : (m < 12) ? d1.y : (m < 14) ? d1.z : d1.w;
              esum += e_at<EXACT>(v.E, id[m], (int)(int16_t)(word >> (16 * (m & 1))));
            }
          } else {
            const uint4 dd = dl4[j];
  #pragma unroll
            for (int m = 1; m < 16; ++m) {
              if (m >= M) break;
              const uint32_t word = (m < 4) ? dd.x : (m < 8) ? dd.y : (m < 12) ? dd.z : dd.w;
              esum += e_at<EXACT>(v.E, id[m], (int)((word >> (8 * (m & 3))) & 0xffu));
            }
          }
          int rk = D - 1 - esum;
          if ((unsigned)rk >= (unsigned)D) {
            atomicOr(a.status, 1);
            rk = 0;
          }
          const float4 gf = Gf[j];
          const dfl cr = SIM ? df_mul_f(dfl{gf.x, gf.y}, Af) : df_mul(dfl{gf.x, gf.y}, AB);
  #pragma unroll
          for (int b = 0; b < B; ++b) {
            const float4 x = gather<LOCAL>(vsec + (size_t)b * total + rk);
            const f2 xh = f2_pack(x.x, x.y), xl = f2_pack(x.z, x.w);
            dfc_fma(acc[b], f2_pack(cr.h, cr.h), f2_pack(-cr.h, -cr.h), f2_pack(cr.l, cr.l), xh, xl);
            if (CPLX) {
              // + (-c_i x_im, c_i x_re): lanes of x swapped, coefficient (-c_i, c_i)
              const dfl ci = SIM ? df_mul_f(dfl{gf.z, gf.w}, Af) : df_mul(dfl{gf.z, gf.w}, AB);
              dfc_fma(acc[b], f2_pack(-ci.h, ci.h), f2_pack(ci.h, -ci.h), f2_pack(-ci.l, ci.l),
                      f2_pack(x.y, x.x), f2_pack(x.w, x.z));
            }
          }
        }
      }
      // keep |lo| below an ulp of hi between pairs
#pragma unroll
      for (int b = 0; b < B; ++b) acc[b] = dfc_renorm(acc[b]);
    }

    const float4 dg4 = a.diag[gr];
    const dfl zf{a.zf.x, a.zf.y};
    // the ket weight where true values are formed (weighted basis)
    const double2 wk = (SIM && (BIL || mode == 1 || mode == 3)) ? ket_weight<MT>(t, occ, kWarpRows)
                                                                 : make_double2(1.0, 1.0);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      dfl acc_r, acc_i;
      f2_unpack(acc[b].h, acc_r.h, acc_i.h);
      f2_unpack(acc[b].l, acc_r.l, acc_i.l);
      const dfl sc{a.scale[b].x, a.scale[b].y};
      const dfl dg = df_add(dfl{dg4.x, dg4.y}, df_mul(sc, dfl{dg4.z, dg4.w}));
      const float4 xo = a.vin[(size_t)b * total + ri];
      const dfl hr = df_add(df_mul(dg, df_re(xo)), df_mul(sc, acc_r));
      const dfl hi = df_add(df_mul(dg, df_im(xo)), df_mul(sc, acc_i));
      if (BIL && mode == 4) {  // <x|H|x>: Re(conj(x) Hx) of this row, no output
        bil_l = df_add(bil_l, df_add(df_mul(df_re(xo), hr), df_mul(df_im(xo), hi)));
        continue;
      }
      if (BIL && b == 0) {
        // H_L x (two-body part at scale 1) and the pair vector of this row
        const float4 pp = a.pair[ri];
        dfl lr = df_add(df_mul(dfl{dg4.z, dg4.w}, df_re(xo)), acc_r);
        dfl li = df_add(df_mul(dfl{dg4.z, dg4.w}, df_im(xo)), acc_i);
        dfl pr = df_re(pp), pi = df_im(pp), xr = df_re(xo), xi = df_im(xo);
        if (SIM) {  // true values: each factor times w (w^2 alone may leave the fp32 range)
          const dfl wd = df_of(wk.x);
          lr = df_mul(wd, lr);
          li = df_mul(wd, li);
          pr = df_mul(wd, pr);
          pi = df_mul(wd, pi);
          xr = df_mul(wd, xr);
          xi = df_mul(wd, xi);
        }
        // Im(conj(p) h) = p.re h.im - p.im h.re
        bil_l = df_add(bil_l, df_add(df_mul(pr, li), df_neg(df_mul(pi, lr))));
        // Im(conj(x) p) = x.re p.im - x.im p.re, weighted by each occupation
        const dfl tx = df_add(df_mul(xr, pi), df_neg(df_mul(xi, pr)));
#pragma unroll
        for (int q = 0; q < kMB; ++q) {
          if (q >= M) break;
          bil_w[q] = df_add(bil_w[q], df_mul(dfl{(float)occ[q * kWarpRows], 0.f}, tx));
        }
      }
      if (mode == 0 || mode == 2) {
        dfl orr = df_mul(zf, hi), oi = df_neg(df_mul(zf, hr));  // z H x with z = -i zre
        if (mode == 0) {
          const float4 p0 = a.psif[(size_t)b * total + ri];
          orr = df_add(df_re(p0), orr);
          oi = df_add(df_im(p0), oi);
        }
        a.out[(size_t)b * total + ri] = df_pack(orr, oi);
      } else if (SIM) {  // modes 1 and 3: back to the FP64 vector, one weight per ket
        double sr = a.zre * df_to(hi), si = -a.zre * df_to(hr);
        if (mode == 3) {
          for (int k = 0; k < a.nbasef; ++k) {
            const float4 e = a.basef[k][(size_t)b * total + ri];
            sr += df_to(df_re(e));
            si += df_to(df_im(e));
          }
        }
        const double2 p0 = a.psi[(size_t)b * total + ri];
        const double nr = p0.x + wk.x * sr, ni = p0.y + wk.x * si;
        a.psi[(size_t)b * total + ri] = make_double2(nr, ni);
        a.out[(size_t)b * total + ri] = df_pack(df_of(nr * wk.y), df_of(ni * wk.y));
      } else {
        const double2 p0 = a.psi[(size_t)b * total + ri];
        double nr = p0.x + a.zre * df_to(hi);
        double ni = p0.y - a.zre * df_to(hr);
        if (mode == 3) {
          for (int k = 0; k < a.nbasef; ++k) {
            const float4 e = a.basef[k][(size_t)b * total + ri];
            nr += df_to(df_re(e));
            ni += df_to(df_im(e));
          }
        }
        a.psi[(size_t)b * total + ri] = make_double2(nr, ni);
        a.out[(size_t)b * total + ri] = df_pack(df_of(nr), df_of(ni));
      }
    }
  }
  __syncwarp();  // the tile's scratch is rewritten by the next tile
}

// Shared-memory view of a stage CTA: the table image (from the ranking table on)
// and the per-warp tile scratch; sets up every pointer stage_tile needs.
struct StageSmem {
  View v;
  const float2* sqf;
  const float4* Gf;
  const uint4* dl4;
  int32_t* sidx;
  uint8_t* socc;
  int32_t* sD;
  int64_t* sOff;
  uint8_t* sperm;
  int32_t* hist;
  int32_t* cursor;
  unsigned char* after;  // first byte after every warp's scratch
};

// Stages the table image (a CTA-wide barrier) and lays out the warp scratch.
template <bool EXACT>
__device__ __forceinline__ StageSmem stage_smem(const Tables& t, unsigned char* smem_raw, int M, int warps) {
  StageSmem S;
  const int from = kSmemFrom(t, EXACT);
  load_blob_from(t, smem_raw, from);
  unsigned char* smem = smem_raw - from;
  S.v = view_at(t, smem);
  if (EXACT) S.v.E = reinterpret_cast<const int32_t*>(t.blob + t.o_E);
  S.sqf = reinterpret_cast<const float2*>(smem + t.o_sqf);
  S.Gf = reinterpret_cast<const float4*>(smem + t.o_Gf);
  S.dl4 = reinterpret_cast<const uint4*>(S.v.delta);
  const int warp = threadIdx.x >> 5;
  const size_t wbytes = df_warp_scratch_bytes(M, t.n_ann);
  unsigned char* base = smem_raw + ((t.blob_bytes - from + 15) & ~15);
  unsigned char* sp = base + (size_t)warp * wbytes;
  S.sidx = reinterpret_cast<int32_t*>(sp);
  S.socc = reinterpret_cast<uint8_t*>(S.sidx + M * kWarpRows);
  S.sD = reinterpret_cast<int32_t*>(S.socc + ((M * kWarpRows + 15) & ~15));
  S.sOff = reinterpret_cast<int64_t*>(S.sD + kWarpRows);
  S.sperm = reinterpret_cast<uint8_t*>(S.sOff + kWarpRows);
  S.hist = reinterpret_cast<int32_t*>(S.sperm + kWarpRows);
  S.cursor = S.hist + (t.n_ann + 2);
  S.after = base + (size_t)warps * wbytes;
  return S;
}

template <int MT, int B, bool CPLX, bool BIL, bool SIM, bool EXACT>
__global__ void __launch_bounds__(kStageBlock, (B == 1 && !BIL) ? kStageMinBlocks : ((BIL && MT > 0) ? 2 : 1))
    stage_df_kernel(const Tables t, const DfArgs a, const int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = (MT > 0) ? MT : t.M;
  // the only CTA-wide barrier: warps run independently afterwards
  const StageSmem S = stage_smem<EXACT>(t, smem_raw, M, kStageWarps);
  constexpr int kWarps = kStageWarps;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row1 = a.row1;
  constexpr int kMB = (MT > 0) ? MT : 16;  // bilinear accumulators: one per mode + H_L
  dfl bil_l{0.f, 0.f};
  dfl bil_w[BIL ? kMB : 1];
#pragma unroll
  for (int q = 0; q < (BIL ? kMB : 1); ++q) bil_w[q] = dfl{0.f, 0.f};

  for (int64_t base = a.row0 + ((int64_t)blockIdx.x * kWarps + warp) * kWarpRows; base < row1;
       base += (int64_t)gridDim.x * kWarps * kWarpRows)
    stage_tile<MT, B, CPLX, BIL, false, SIM, EXACT>(t, S.v, S.sqf, S.Gf, S.dl4, a, mode, base, row1, 0, S.sidx, S.socc,
                                             S.sD, S.sOff, S.sperm, S.hist, S.cursor, bil_l, bil_w);
  if (BIL) {
    // per-CTA sums of the bilinears in a fixed order: lanes by shuffles, warps in turn
    __shared__ double red[kStageWarps][17];
    const int nq = M + 1;
    for (int q = 0; q < nq; ++q) {
      double v = (q == 0) ? df_to(bil_l) : 0.0;
#pragma unroll
      for (int u = 0; u < kMB; ++u)
        if (q == u + 1) v = df_to(bil_w[u]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += red[w][threadIdx.x];
      a.partial[(size_t)blockIdx.x * nq + threadIdx.x] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// Resident small sectors: each CTA takes sectors [0, n_small) from a static work
// list (sector c, c + gridDim.x, ...), copies the sector's psi into shared
// memory and runs all `steps` RK4 steps there, with only CTA barriers between
// stages -- the sectors are independent, so no CTA ever waits on another.  The
// final psi and its double-float copy are written back to global memory.
struct ResArgs {
  double2* psi;        // global psi [total]
  float4* psif;        // global double-float copy of psi in the weighted basis [total] (read, written back)
  const float4* diag;  // per-ket diagonal
  float2 scale;        // two-body scale, double-float
  double dt;
  int64_t steps;
  int order;           // Taylor order of a step (stages per step)
  int n_small;         // sectors [0, n_small) are resident
  int cap;             // kets per sector the shared buffers hold
  int* status;
};

template <int MT, bool CPLX, bool EXACT>
__global__ void __launch_bounds__(kBlock) resident_kernel(const Tables t, const ResArgs r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = (MT > 0) ? MT : t.M;
  const StageSmem S = stage_smem<EXACT>(t, smem_raw, M, kBlock / 32);
  double2* spsi = reinterpret_cast<double2*>(S.after);
  float4* spsif = reinterpret_cast<float4*>(spsi + r.cap);
  float4* sw1 = spsif + r.cap;
  float4* sw2 = sw1 + r.cap;
  constexpr int kWarps = kBlock / 32;
  const int warp = threadIdx.x >> 5;
  dfl bil_l{0.f, 0.f}, bil_w[1] = {dfl{0.f, 0.f}};
  for (int sid = blockIdx.x; sid < r.n_small; sid += gridDim.x) {
    const int64_t off = __ldg(t.sec_off + sid);
    const int D = (int)(__ldg(t.sec_off + sid + 1) - off);
    if (D > r.cap) {  // not reached: the host lists only sectors that fit
      if (threadIdx.x == 0) atomicOr(r.status, 4);
      continue;
    }
    for (int i = threadIdx.x; i < D; i += kBlock) {
      spsi[i] = r.psi[off + i];
      spsif[i] = r.psif[off + i];  // the weighted double-float copy
    }
    __syncthreads();
    DfArgs a{};
    a.diag = r.diag;
    a.scale[0] = r.scale;
    a.status = r.status;
    a.psi = spsi;
    a.psif = spsif;
    a.nbasef = 0;
    for (int64_t it = 0; it < r.steps; ++it) {
      for (int d = r.order; d >= 1; --d) {
        const int j = r.order - d;
        a.vin = (j == 0) ? spsif : ((j - 1) % 2 == 0 ? sw1 : sw2);
        a.out = (d == 1) ? spsif : (j % 2 == 0 ? sw1 : sw2);
        a.zre = r.dt / d;
        const float zh = (float)a.zre;
        a.zf = make_float2(zh, (float)(a.zre - (double)zh));
        // the sector's kets are dealt to the warps in chunks of at most kWarpRows,
        // evenly, so that a small sector still keeps every warp busy
        const int64_t chunk = min((int64_t)kWarpRows, ((int64_t)D + kWarps - 1) / kWarps);
        for (int64_t base = off + (int64_t)warp * chunk; base < off + D; base += (int64_t)kWarps * chunk)
          stage_tile<MT, 1, CPLX, false, true, true, EXACT>(t, S.v, S.sqf, S.Gf, S.dl4, a, d == 1 ? 1 : 0, base,
                                               min(base + chunk, off + (int64_t)D), off, S.sidx, S.socc, S.sD,
                                               S.sOff, S.sperm, S.hist, S.cursor, bil_l, bil_w);
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < D; i += kBlock) {
      r.psi[off + i] = spsi[i];
      r.psif[off + i] = spsif[i];
    }
    __syncthreads();
  }
}

// Shared memory of the resident kernel holding `cap` kets per sector.
inline size_t resident_smem(const Tables& t, int cap) {
  return ((t.blob_bytes - kSmemFrom(t, t.exact != 0) + 15) & ~15) + df_scratch_bytes(t.M, t.n_ann) +
         (size_t)cap * 64;
}

template <int MT, bool EXACT>
int resident_launch_e(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  const size_t smem = resident_smem(t, r.cap);
  int grid = 0, rc = QB_OK;
  if (cplx) {
    auto k = resident_kernel<MT, true, EXACT>;
    rc = persistent_grid(k, smem, (int64_t)r.n_small * kBlock, &grid);
    if (rc) return rc;
    k<<<grid, kBlock, smem, st>>>(t, r);
  } else {
    auto k = resident_kernel<MT, false, EXACT>;
    rc = persistent_grid(k, smem, (int64_t)r.n_small * kBlock, &grid);
    if (rc) return rc;
    k<<<grid, kBlock, smem, st>>>(t, r);
  }
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

template <int MT>
int resident_launch_t(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  if (t.exact) return resident_launch_e<MT, true>(t, r, cplx, st);
  return resident_launch_e<MT, false>(t, r, cplx, st);
}

// Launches one stage for mode count MT (0: any M) and the runtime batch size /
// coupling type / bilinear flag / basis (sim: the weighted basis of the RK4 and
// adjoint stages, modes 0 to 3; plain: the <H> reduction, mode 4); *grid (if
// non-NULL) receives the grid size.  Exact momentum: one state at a time.
template <int MT, bool EXACT>
int stage_launch_e(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, bool bil, bool sim, cudaStream_t st,
                   int* grid_out) {
  const size_t smem = ((t.blob_bytes - kSmemFrom(t, EXACT) + 15) & ~15) +
                      (size_t)kStageWarps * df_warp_scratch_bytes(t.M, t.n_ann);
  int grid = 0, rc = QB_OK;
#define QB_STAGE_CASE(BB, CC, LL, SS)                                           \
  {                                                                             \
    auto k = stage_df_kernel<MT, BB, CC, LL, SS, EXACT>;                        \
    rc = persistent_grid(k, smem, a.row1 - a.row0, &grid, kStageBlock);         \
    if (rc) return rc;                                                          \
    k<<<grid, kStageBlock, smem, st>>>(t, a, mode);                             \
  }
  if (sim) {
    if (mode < 0 || mode > 3) return fail(QB_EINTERNAL, "the weighted basis serves modes 0 to 3");
    if (bil) {
      if (B != 1) return fail(QB_EUNSUPPORTED, "bilinear stages run one state at a time");
      if (cplx)
        QB_STAGE_CASE(1, true, true, true)
      else
        QB_STAGE_CASE(1, false, true, true)
    } else if (cplx) {
      if (B != 1) return fail(QB_EUNSUPPORTED, "batched sweeps need a real coupling");
      QB_STAGE_CASE(1, true, false, true)
    } else {
      if constexpr (EXACT) {
        if (B != 1) return fail(QB_EUNSUPPORTED, "exact momentum: batched sweeps are not built");
        QB_STAGE_CASE(1, false, false, true)
      } else {
        switch (B) {
          case 1: QB_STAGE_CASE(1, false, false, true) break;
          case 2: QB_STAGE_CASE(2, false, false, true) break;
          case 4: QB_STAGE_CASE(4, false, false, true) break;
          case 8: QB_STAGE_CASE(8, false, false, true) break;
          default: return fail(QB_EINVAL, "batch must be 1, 2, 4 or 8");
        }
      }
    }
  } else {
    // the plain basis serves the <x|H|x> reduction of the observables
    if (!bil || mode != 4 || B != 1) return fail(QB_EINTERNAL, "the plain basis serves the <H> reduction only");
    if (cplx)
      QB_STAGE_CASE(1, true, true, false)
    else
      QB_STAGE_CASE(1, false, true, false)
  }
#undef QB_STAGE_CASE
  QB_CUDA(cudaGetLastError());
  if (grid_out) *grid_out = grid;
  return QB_OK;
}

template <int MT>
int stage_launch_t(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, bool bil, bool sim, cudaStream_t st,
                   int* grid_out) {
  if (t.exact) return stage_launch_e<MT, true>(t, a, mode, B, cplx, bil, sim, st, grid_out);
  return stage_launch_e<MT, false>(t, a, mode, B, cplx, bil, sim, st, grid_out);
}

// one explicit specialisation per translation unit (qb_stage_m*.cu)
int stage_launch_m5(const Tables&, const DfArgs&, int, int, bool, bool, bool, cudaStream_t, int*);
int stage_launch_m7(const Tables&, const DfArgs&, int, int, bool, bool, bool, cudaStream_t, int*);
int stage_launch_m9(const Tables&, const DfArgs&, int, int, bool, bool, bool, cudaStream_t, int*);
int stage_launch_m11(const Tables&, const DfArgs&, int, int, bool, bool, bool, cudaStream_t, int*);
int stage_launch_any(const Tables&, const DfArgs&, int, int, bool, bool, bool, cudaStream_t, int*);

int resident_launch_m5(const Tables&, const ResArgs&, bool, cudaStream_t);
int resident_launch_m7(const Tables&, const ResArgs&, bool, cudaStream_t);
int resident_launch_m9(const Tables&, const ResArgs&, bool, cudaStream_t);
int resident_launch_m11(const Tables&, const ResArgs&, bool, cudaStream_t);
int resident_launch_any(const Tables&, const ResArgs&, bool, cudaStream_t);

inline int resident_launch(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  switch (t.M) {
    case 5: return resident_launch_m5(t, r, cplx, st);
    case 7: return resident_launch_m7(t, r, cplx, st);
    case 9: return resident_launch_m9(t, r, cplx, st);
    case 11: return resident_launch_m11(t, r, cplx, st);
    default: return resident_launch_any(t, r, cplx, st);
  }
}

inline int stage_launch(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, cudaStream_t st,
                        int* grid_out = nullptr, bool bil = false, bool sim = false) {
  switch (t.M) {
    case 5: return stage_launch_m5(t, a, mode, B, cplx, bil, sim, st, grid_out);
    case 7: return stage_launch_m7(t, a, mode, B, cplx, bil, sim, st, grid_out);
    case 9: return stage_launch_m9(t, a, mode, B, cplx, bil, sim, st, grid_out);
    case 11: return stage_launch_m11(t, a, mode, B, cplx, bil, sim, st, grid_out);
    default: return stage_launch_any(t, a, mode, B, cplx, bil, sim, st, grid_out);
  }
}

}  // namespace qb
