// The hot kernel: one Horner RK4 stage of every sector (and every member of a
// batched coupling sweep) in one launch, with the matrix-free sector H psi in
// double-float arithmetic, in the weighted basis f = psi / w(n).
//
//   stage d (d = 4, 3, 2):  out = f + (-i dt/d) W^-1 H W v    (double-float out)
//   stage 1:                psi = psi + (-i dt) H v, f = psi / w
//                                                     (FP64 psi, plus its weighted copy)
//
// H is Eq. (Ham) restricted to sectors of fixed N and momentum mod M (Sec. III B).
// Per row (ket n) the off-diagonal terms are the disjoint pairs {r, s} -> {p, q}
// with p + q = r + s (mod M); in the weighted basis, w(n) = sqrt(N! / prod n_m!) up
// to a power of two per N, the element of target n' = n - e_r - e_s + e_p + e_q is
// G_{pq,rs} n_r (n_s - [r = s]): the ratio w(n') / w(n) cancels the creation
// square roots and squares the annihilation ones.  G is the multiplicity-summed
// symmetrised coupling; the diagonal is precomputed per ket.
//
// Work layout: every warp owns tiles of kRows consecutive kets and runs without
// CTA-wide barriers.  Phase 1 unpacks the tile's occupations (kRows/32 kets per
// lane) and their suffix-state indices; phase 2 counting-sorts the tile by the
// number of annihilation pairs acting on each ket; phase 3 runs the terms in
// rounds, the 32 lanes of a round taking 32 kets of nearly equal work.  For odd M
// every annihilation pair has exactly (M-1)/2 creation partners; the specialised
// kernels unroll them so that their ranks and gathers overlap.
//
// Ranking (RK): a target's rank is D - 1 - sum_{m=1}^{M-1} E[idx_m + shift_m], the
// shift of the suffix index at mode m fixed by the term.
//   RK_PAIR   momentum mod M: the ranking table sits in shared memory and spans
//             < 64 KB (qb_sector_build refuses larger ones), so the byte offsets of
//             modes 2k+1 and 2k+2 share one 32-bit word per ket, and one 32-bit add
//             of the term's packed shifts advances both (the shifts are stored as the
//             signed value lo + 65536 hi, so the low half's borrow is part of it);
//   RK_EXACT  exact momentum: 16-bit shifts, the ranking table in global memory.
#pragma once
#include "qb_device.cuh"

#ifndef QB_UNROLL_PARTNERS
#define QB_UNROLL_PARTNERS 1
#endif
// 1: the specialised kernels for odd M <= QB_REG_OCC_MAX_M take a pair's occupations
// from registers
#ifndef QB_REG_OCC
#define QB_REG_OCC 1
#endif
#ifndef QB_REG_OCC_MAX_M
#define QB_REG_OCC_MAX_M 11
#endif
// 1: a ket's sector from its occupations (N, K) and the (N, K) -> sector table;
// 0: binary search of the sector offsets
#ifndef QB_SEC_FROM_WORD
#define QB_SEC_FROM_WORD 1
#endif

namespace qb {

enum { RK_PAIR = 1, RK_EXACT = 2 };

// n_m of occupations held as bytes in three words (modes 0-3, 4-7, 8-11)
template <int MT>
__device__ __forceinline__ int reg_occ(uint32_t ob0, uint32_t ob1, uint32_t ob2, int m) {
  if constexpr (MT <= 8) return (int)(__byte_perm(ob0, ob1, (uint32_t)m) & 0xffu);
  return m < 8 ? (int)(__byte_perm(ob0, ob1, (uint32_t)m) & 0xffu) : (int)((ob2 >> (8 * (m - 8))) & 0xffu);
}

// What a stage launch computes besides (or instead of) its output vector:
//   KIND_STAGE  the RK4 / adjoint stage alone (modes 0 to 3);
//   KIND_BIL    with the adjoint's bilinears fused (modes 2, 3);
//   KIND_DOT    <x|H|x> only (mode 4): Re(conj(psi_n) (H psi)_n) summed in FP64,
//               with each off-diagonal term and its Hermitian reverse taken once
//               (the partners of a pair that come after it, counted twice).
enum { KIND_STAGE = 0, KIND_BIL = 1, KIND_DOT = 2 };

// Tile shapes of the stage kernel: warps per CTA, kets per warp tile and the
// resident CTAs per SM its register budget is planned for (65,536 registers per SM
// shared by warps x 32 x CTAs threads).  The CTA's warps share one copy of the
// ranking table in shared memory.  Shape 0 is the default; the others are
// compiled for the single-state stage (qb_space_set_tile_shape selects one).
struct TileShape {
  int warps, rows, min_blocks;
};
constexpr int kTileShapes = 5;
__host__ __device__ constexpr TileShape tile_shape(int ts) {
  return ts == 1   ? TileShape{16, 64, 2}
         : ts == 2 ? TileShape{24, 64, 1}
         : ts == 3 ? TileShape{12, 64, 3}
         : ts == 4 ? TileShape{32, 128, 1}
                   : TileShape{32, 64, 1};
}
// the shape of the batched sweeps and the bilinear stages (12 warps: room for the
// registers of their extra accumulators)
constexpr int kWideShape = 3;

// Shared scratch of the stage kernel, after the table image, per warp (a tile of
// `rows` kets):
//   sidx  int32 [iw][rows]  suffix-state offsets of each ket: RK_PAIR two modes per
//                           word (iw = M/2 words), RK_EXACT one per mode (iw = M)
//   socc  uint8 [M][rows]   occupations
//   sD    int32 [rows]      sector dimension of the ket (-1: no ket)
//   sOff  int64 [rows]      sector offset of the ket
//   sperm uint8 [rows]      processing order (kets sorted by work, most first)
//   hist  int32 [2][n_ann+2] counting-sort buckets and cursors
__host__ __device__ inline int sidx_words(int M, bool exact) { return exact ? M : (M / 2 > 0 ? M / 2 : 1); }
__host__ __device__ inline size_t df_warp_scratch_bytes(int iw, int M, int n_ann, int rows) {
  size_t b = (size_t)iw * rows * 4 + (((size_t)M * rows + 15) & ~(size_t)15);
  b += (size_t)rows * 4 + (size_t)rows * 8 + rows + 2 * (size_t)(n_ann + 2) * 4;
  return (b + 15) & ~(size_t)15;
}

// The bytes [kSmemFrom, kSmemEnd) of the table image the stage kernels stage in
// shared memory: the ranking table (mod M; exact momentum keeps it in global
// memory), the pair offsets and indices, the couplings and the term shifts (exact
// momentum: the int16 shift table)
__host__ __device__ inline int kSmemFrom(const Tables& t, bool exact = false) { return exact ? t.o_Ex : t.o_E; }
__host__ __device__ inline int kSmemEnd(const Tables& t, bool exact = false) { return exact ? t.o_sqrt : t.o_delta; }

// Gathered stage-vector entry: read-only global load, or a generic load when the
// vector is a shared-memory copy (LOCAL; the non-coherent global path does not
// accept shared addresses).
template <bool LOCAL>
__device__ __forceinline__ float4 gather(const float4* p) {
  if (LOCAL) return *p;
  return __ldg(p);
}

// The stage kernels' dynamic shared memory: the table image from the ranking table
// on (non-exact momentum), so a byte offset into the ranking table is one shared
// load with an immediate base.
extern __shared__ __align__(16) unsigned char stage_smem_raw[];
__device__ __forceinline__ int32_t e_byte(uint32_t off) {
  return *reinterpret_cast<const int32_t*>(stage_smem_raw + off);
}

// sum_{m=1}^{M-1} E[idx_m + shift_m] of combo j for a ket whose suffix indices are
// id[] (RK_PAIR: packed byte offsets, two modes per word; RK_EXACT: byte offsets
// per mode)
template <int MT, int RK>
__device__ __forceinline__ int rank_esum(const Tables& t, const int32_t* E, const unsigned char* dtab, int j,
                                         const int* id) {
  const int M = (MT > 0) ? MT : t.M;
  int esum = 0;
  if constexpr (RK == RK_PAIR) {
    // words 0 and 1 side by side, word k >= 2 in column k of the ncp-row table
    const uint2 w01 = reinterpret_cast<const uint2*>(dtab)[j];
    const uint32_t* wk = reinterpret_cast<const uint32_t*>(dtab) + j;
    constexpr int kW = (MT > 0) ? MT / 2 : 8;
#pragma unroll
    for (int k = 0; k < kW; ++k) {
      if (MT == 0 && 2 * k + 1 >= M) break;
      const uint32_t dk = (k == 0) ? w01.x : (k == 1) ? w01.y : wk[(size_t)k * t.ncp];
      const uint32_t u = (uint32_t)id[k] + dk;
      esum += e_byte(u & 0xffffu);
      // the high half of the last word is mode M when M is even: offset 0, where
      // the table holds zero (mode 0, fewer than one particle)
      if (MT == 0 || 2 * k + 2 < MT) esum += e_byte(u >> 16);
    }
  } else {  // RK_EXACT: int16 shifts, two modes per word (modes 8-15 in the second row)
    const uint4 d0 = reinterpret_cast<const uint4*>(dtab)[2 * (size_t)j];
    uint4 d1 = make_uint4(0u, 0u, 0u, 0u);
    if (MT == 0 || MT > 8) d1 = reinterpret_cast<const uint4*>(dtab)[2 * (size_t)j + 1];
#pragma unroll
    for (int m = 1; m < 16; ++m) {
      if (m >= M) break;
      const uint32_t word = (m < 2) ? d0.x : (m < 4) ? d0.y : (m < 6) ? d0.z : (m < 8) ? d0.w
                          : (m < 10) ? d1.x : (m < 12) ? d1.y : (m < 14) ? d1.z : d1.w;
      const int sh = (int)(int16_t)(word >> (16 * (m & 1))) << 2;
      if (t.ex_smem)  // the compact table staged in shared memory
        esum += e_byte((uint32_t)(id[m] + sh));
      else  // the ranking table is read-only for the kernel's life: the non-coherent path
        esum += __ldg(reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(E) + id[m] + sh));
    }
  }
  return esum;
}

// One warp tile: kets [base, min(base + kRows, row1)) of the launch.  With LOCAL
// the state vectors of DfArgs are the shared-memory copies of one sector starting
// at ket local_off (gathers and own-row accesses are sector-local); otherwise they
// are the global vectors.  The per-ket diagonal is always global.
//
// The double-float vectors hold f = psi / w; modes 1 and 3 map back to the FP64
// vector: psi += w (z W^-1 H W f + sum of basef), and write f = psi_new / w; the
// bilinears and the <x|H|x> reduction multiply by w where true values are formed.
//
// A gather index outside its sector is clamped into it and flagged in the status
// word once per ket (bit 0), without a branch per term.
template <int MT, int B, bool CPLX, int KIND, bool LOCAL, int RK, int kRows>
__device__ __forceinline__ void stage_tile(const Tables& t, const View& v, const float2* Gf, const unsigned char* dtab,
                                           const DfArgs& a, const int mode, const int64_t base, const int64_t row1,
                                           const int64_t local_off, int32_t* sidx, uint8_t* socc, int32_t* sD,
                                           int64_t* sOff, uint8_t* sperm, int32_t* hist, int32_t* cursor, dfl& bil_l,
                                           dfl* bil_w, double& dot64) {
  constexpr bool EXACT = (RK == RK_EXACT);
  constexpr bool BIL = (KIND == KIND_BIL), DOT = (KIND == KIND_DOT);
  const int M = (MT > 0) ? MT : t.M;
  const int Qm = EXACT ? t.Q : M;  // momentum modulus
  const int twoM = 2 * Qm;         // row width of the ranking table
  const int lane = threadIdx.x & 31;
  const int64_t total = t.total;  // stride between sweep members
  const int nb = t.n_ann + 2;
  constexpr int kMB = (MT > 0) ? MT : 16;
  constexpr int kPW = (MT > 0) ? (MT / 2 > 0 ? MT / 2 : 1) : 8;  // packed index words (RK_PAIR)
  // ---- phase 1: each lane unpacks kRows/32 kets into occupations and suffix-state indices
  for (int k = lane; k < 2 * nb; k += 32) hist[k] = 0;
  int key[kRows / 32];
#pragma unroll
  for (int u = 0; u < kRows / 32; ++u) {
    const int row = u * 32 + lane;
    const int64_t g = base + row;
    key[u] = 0;
    if (g < row1) {
      const uint64_t word = __ldg(t.occ + g);
      const int ob = t.occ_bits;
      int nN = 0, nK = 0;
      for (int m = 0; m < M; ++m) {
        const int nm = occ_of(word, m, ob);
        socc[m * kRows + row] = (uint8_t)nm;
        nN += nm;
        nK += m * nm;
      }
#if QB_SEC_FROM_WORD
      const int sid = __ldg(t.sec_of + nN * Qm + nK % Qm);
#else
      const int sid = find_sector(t, g);
#endif
      const int64_t off = __ldg(t.sec_off + sid);
      const int D = (int)(__ldg(t.sec_off + sid + 1) - off);
      int srem = 0, skr = 0, esum = 0, np = 0, n2 = 0;
      uint32_t pk[kPW];
#pragma unroll
      for (int k = 0; k < kPW; ++k) pk[k] = 0u;
      for (int m = M - 1; m >= 1; --m) {
        const int nm = socc[m * kRows + row];
        srem += nm;
        skr += m * nm;
        while (skr >= Qm) skr -= Qm;
        const int ix = (m * t.rem_w + srem + 2) * twoM + skr;
        if (EXACT && t.ex_smem) {  // byte offset into the compact table (column skr - m srem)
          const int ixb = t.ex_base[m] + ((srem + 2) * t.ex_w[m] + skr - m * srem) * 4;
          esum += e_byte((uint32_t)ixb);
          sidx[m * kRows + row] = ixb;
          continue;
        }
        esum += v.E[ix];
        if constexpr (RK == RK_PAIR) {
#pragma unroll
          for (int k = 0; k < kPW; ++k)
            if (k == ((m - 1) >> 1)) pk[k] |= (uint32_t)(ix * 4) << ((m & 1) ? 0 : 16);
        } else {
          sidx[m * kRows + row] = ix * 4;
        }
      }
      if constexpr (RK == RK_PAIR) {
#pragma unroll
        for (int k = 0; k < kPW; ++k)
          if (2 * k + 1 < M) sidx[k * kRows + row] = (int32_t)pk[k];
      }
      if (D - 1 - esum != (int)(g - off)) atomicOr(a.status, 2);
      for (int m = 0; m < M; ++m) {
        const int nm = socc[m * kRows + row];
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
  for (int u = 0; u < kRows / 32; ++u) atomicAdd(&hist[key[u]], 1);
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
  for (int u = 0; u < kRows / 32; ++u) sperm[atomicAdd(&cursor[key[u]], 1)] = (uint8_t)(u * 32 + lane);
  __syncwarp();

  // ---- phase 3: rounds of 32 kets of similar work, one per lane
  for (int round = 0; round < kRows / 32; ++round) {
    const int row = sperm[round * 32 + lane];
    const int D = sD[row];
    if (D < 0) continue;
    const int64_t off = sOff[row];
    const int64_t gr = base + row;
    const int64_t ri = LOCAL ? gr - local_off : gr;  // own-row index into the state vectors
    const uint8_t* occ = socc + row;
    int id[16];
    if constexpr (RK == RK_PAIR) {
#pragma unroll
      for (int k = 0; k < kPW; ++k)
        if (2 * k + 1 < M) id[k] = sidx[k * kRows + row];
    } else {
#pragma unroll
      for (int m = 1; m < 16; ++m)
        if (m < M) id[m] = sidx[m * kRows + row];
    }
    uint32_t occmask = 0, twomask = 0;
    // the specialised odd-M kernels with M <= 7 also keep the occupations as bytes in
    // registers, so that a pair's n_r and n_s are byte permutes instead of shared loads
    constexpr bool kRegOcc =
        QB_REG_OCC && MT > 0 && MT <= QB_REG_OCC_MAX_M && (MT % 2) == 1 && !CPLX && !EXACT && !DOT;
    uint32_t ob0 = 0u, ob1 = 0u, ob2 = 0u;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (m >= M) break;
      const int nm = occ[m * kRows];
      occmask |= (nm >= 1 ? 1u : 0u) << m;
      twomask |= (nm >= 2 ? 1u : 0u) << m;
      if (kRegOcc) {
        if (m < 4)
          ob0 |= (uint32_t)nm << (8 * m);
        else if (m < 8)
          ob1 |= (uint32_t)nm << (8 * (m - 4));
        else
          ob2 |= (uint32_t)nm << (8 * (m - 8));
      }
    }
    const float4* vsec = a.vin + (LOCAL ? 0 : off);  // gathers
    dfc acc[B];  // (re, im) of the off-diagonal sum, double-float, packed
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = dfc{0ull, 0ull};
    bool bad = false;  // a target rank fell outside the sector

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
      const int s = __ffs(smask) - 1;
      smask &= smask - 1;
      // pair index of (r <= s) in the order r = 0.., s = r..: r (2M - r + 1) / 2 + s - r
      const int ai = kRegOcc ? (r * (2 * MT - r + 1)) / 2 + s - r : v.pairidx[r * 16 + s];
      const int nr = kRegOcc ? reg_occ<MT>(ob0, ob1, ob2, r) : occ[r * kRows];
      const int ns = kRegOcc ? reg_occ<MT>(ob0, ob1, ob2, s) : occ[s * kRows];
      const float Af = (float)(nr * (ns - (r == s ? 1 : 0)));  // exact
      // (exact momentum: the partner count varies from pair to pair; <x|H|x> takes
      // only the partners after the pair)
      constexpr int kC =
          (QB_UNROLL_PARTNERS && !CPLX && !EXACT && !DOT && MT > 0 && (MT % 2) == 1) ? (MT - 1) / 2 : 0;
      if (kC > 0) {
        // fixed partner count: all ranks first, then all gathers, then the sums
        // every pair has kC partners, laid out pair by pair
        const int j0 = kRegOcc ? ai * kC : v.ann[ai];
        int rkc[kC > 0 ? kC : 1];
        dfl crc[kC > 0 ? kC : 1];
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          const int j = j0 + c;
          const uint32_t rk = (uint32_t)(D - 1 - rank_esum<MT, RK>(t, v.E, dtab, j, id));
          bad |= rk >= (uint32_t)D;
          rkc[c] = (int)min(rk, (uint32_t)(D - 1));
          const float2 gr = Gf[j];  // real coupling (hi, lo)
          crc[c] = df_mul_f(dfl{gr.x, gr.y}, Af);
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
      } else if (DOT && !CPLX && B == 1) {
        // <x|H|x>: the partners after the pair, two terms in flight
        const int j1 = v.ann[ai + 1];
        int j = v.hs[ai];
        for (; j + 1 < j1; j += 2) {
          const uint32_t ra = (uint32_t)(D - 1 - rank_esum<MT, RK>(t, v.E, dtab, j, id));
          const uint32_t rb = (uint32_t)(D - 1 - rank_esum<MT, RK>(t, v.E, dtab, j + 1, id));
          bad |= (ra >= (uint32_t)D) | (rb >= (uint32_t)D);
          const float4 xa = gather<LOCAL>(vsec + min(ra, (uint32_t)(D - 1)));
          const float4 xb = gather<LOCAL>(vsec + min(rb, (uint32_t)(D - 1)));
          const float2 ga = Gf[j], gb = Gf[j + 1];
          const dfl ca = df_mul_f(dfl{ga.x, ga.y}, Af), cb = df_mul_f(dfl{gb.x, gb.y}, Af);
          dfc_fma(acc[0], f2_pack(ca.h, ca.h), f2_pack(-ca.h, -ca.h), f2_pack(ca.l, ca.l), f2_pack(xa.x, xa.y),
                  f2_pack(xa.z, xa.w));
          dfc_fma(acc[0], f2_pack(cb.h, cb.h), f2_pack(-cb.h, -cb.h), f2_pack(cb.l, cb.l), f2_pack(xb.x, xb.y),
                  f2_pack(xb.z, xb.w));
        }
        if (j < j1) {
          const uint32_t ra = (uint32_t)(D - 1 - rank_esum<MT, RK>(t, v.E, dtab, j, id));
          bad |= ra >= (uint32_t)D;
          const float4 xa = gather<LOCAL>(vsec + min(ra, (uint32_t)(D - 1)));
          const float2 ga = Gf[j];
          const dfl ca = df_mul_f(dfl{ga.x, ga.y}, Af);
          dfc_fma(acc[0], f2_pack(ca.h, ca.h), f2_pack(-ca.h, -ca.h), f2_pack(ca.l, ca.l), f2_pack(xa.x, xa.y),
                  f2_pack(xa.z, xa.w));
        }
      } else {
        const int j1 = v.ann[ai + 1];
        for (int j = DOT ? v.hs[ai] : v.ann[ai]; j < j1; ++j) {
          const uint32_t rku = (uint32_t)(D - 1 - rank_esum<MT, RK>(t, v.E, dtab, j, id));
          bad |= rku >= (uint32_t)D;
          const int rk = (int)min(rku, (uint32_t)(D - 1));
          const float2 gr = Gf[j];  // coupling (re.hi, re.lo), (im.hi, im.lo)
          const float2 gi = CPLX ? Gf[t.ncp + j] : make_float2(0.f, 0.f);
          const dfl cr = df_mul_f(dfl{gr.x, gr.y}, Af);
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const float4 x = gather<LOCAL>(vsec + (size_t)b * total + rk);
            const f2 xh = f2_pack(x.x, x.y), xl = f2_pack(x.z, x.w);
            dfc_fma(acc[b], f2_pack(cr.h, cr.h), f2_pack(-cr.h, -cr.h), f2_pack(cr.l, cr.l), xh, xl);
            if (CPLX) {
              // + (-c_i x_im, c_i x_re): lanes of x swapped, coefficient (-c_i, c_i)
              const dfl ci = df_mul_f(dfl{gi.x, gi.y}, Af);
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
    if (bad) atomicOr(a.status, 1);

    const float4 dg4 = a.diag[gr];
    const dfl zf{a.zf.x, a.zf.y};
    // the ket weight where true values are formed
    const double2 wk = (BIL || DOT || mode == 1 || mode == 3) ? ket_weight<MT>(t, occ, kRows) : make_double2(1.0, 1.0);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      dfl acc_r, acc_i;
      f2_unpack(acc[b].h, acc_r.h, acc_i.h);
      f2_unpack(acc[b].l, acc_r.l, acc_i.l);
      if (DOT) {  // each term stands for itself and its reverse (H Hermitian): twice the real part
        acc_r = dfl{2.f * acc_r.h, 2.f * acc_r.l};
        acc_i = dfl{2.f * acc_i.h, 2.f * acc_i.l};
      }
      const dfl sc{a.scale[b].x, a.scale[b].y};
      const dfl dg = df_add(dfl{dg4.x, dg4.y}, df_mul(sc, dfl{dg4.z, dg4.w}));
      const float4 xo = a.vin[(size_t)b * total + ri];
      const dfl hr = df_add(df_mul(dg, df_re(xo)), df_mul(sc, acc_r));
      const dfl hi = df_add(df_mul(dg, df_im(xo)), df_mul(sc, acc_i));
      if (DOT) {
        // <x|H|x>: Re(conj(psi_n) (H psi)_n) = w^2 Re(conj(f_n) (W^-1 H W f)_n), w^2 in
        // FP64 (w^2 alone may leave the fp32 range); no output
        const dfl val = df_add(df_mul(df_re(xo), hr), df_mul(df_im(xo), hi));
        dot64 += df_to(val) * wk.x * wk.x;
        continue;
      }
      if (BIL && b == 0) {
        // H_L x (two-body part at scale 1) and the pair vector of this row, as true
        // values: each factor times w (w^2 alone may leave the fp32 range)
        const float4 pp = a.pair[ri];
        const dfl wd = df_of(wk.x);
        const dfl lr = df_mul(wd, df_add(df_mul(dfl{dg4.z, dg4.w}, df_re(xo)), acc_r));
        const dfl li = df_mul(wd, df_add(df_mul(dfl{dg4.z, dg4.w}, df_im(xo)), acc_i));
        const dfl pr = df_mul(wd, df_re(pp)), pi = df_mul(wd, df_im(pp));
        const dfl xr = df_mul(wd, df_re(xo)), xi = df_mul(wd, df_im(xo));
        // Im(conj(p) h) = p.re h.im - p.im h.re
        bil_l = df_add(bil_l, df_add(df_mul(pr, li), df_neg(df_mul(pi, lr))));
        // Im(conj(x) p) = x.re p.im - x.im p.re, weighted by each occupation
        const dfl tx = df_add(df_mul(xr, pi), df_neg(df_mul(xi, pr)));
#pragma unroll
        for (int q = 0; q < kMB; ++q) {
          if (q >= M) break;
          bil_w[q] = df_add(bil_w[q], df_mul(dfl{(float)occ[q * kRows], 0.f}, tx));
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
      } else {  // modes 1 and 3: back to the FP64 vector, one weight per ket
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
      }
    }
  }
  __syncwarp();  // the tile's scratch is rewritten by the next tile
}

// Shared-memory view of a stage CTA: the table image (from the ranking table on)
// and the per-warp tile scratch; sets up every pointer stage_tile needs.
struct StageSmem {
  View v;
  const float2* Gf;           // coupling columns (real, imaginary) of ncp double-float pairs
  const unsigned char* dtab;  // shifts of the ranking variant
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
template <int RK>
__device__ __forceinline__ StageSmem stage_smem(const Tables& t, int M, int warps, int rows) {
  StageSmem S;
  const int from = kSmemFrom(t, RK == RK_EXACT), end = kSmemEnd(t, RK == RK_EXACT);
  {
    const int4* src = reinterpret_cast<const int4*>(t.blob + from);
    int4* dst = reinterpret_cast<int4*>(stage_smem_raw);
    for (int i = threadIdx.x; i < (end - from) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
  }
  unsigned char* smem = stage_smem_raw - from;
  S.v = view_at(t, smem);
  if (RK == RK_EXACT) S.v.E = reinterpret_cast<const int32_t*>(t.blob + t.o_E);
  S.Gf = reinterpret_cast<const float2*>(smem + t.o_Gf);
  S.dtab = (RK == RK_PAIR) ? smem + t.o_dsw
                           : (t.ex_smem ? smem + t.o_dex : reinterpret_cast<const unsigned char*>(S.v.delta));
  const int warp = threadIdx.x >> 5;
  const int iw = sidx_words(M, RK == RK_EXACT);
  const size_t wbytes = df_warp_scratch_bytes(iw, M, t.n_ann, rows);
  unsigned char* base = stage_smem_raw + ((end - from + 15) & ~15);
  unsigned char* sp = base + (size_t)warp * wbytes;
  S.sidx = reinterpret_cast<int32_t*>(sp);
  S.socc = reinterpret_cast<uint8_t*>(S.sidx + iw * rows);
  S.sD = reinterpret_cast<int32_t*>(S.socc + ((M * rows + 15) & ~15));
  S.sOff = reinterpret_cast<int64_t*>(S.sD + rows);
  S.sperm = reinterpret_cast<uint8_t*>(S.sOff + rows);
  S.hist = reinterpret_cast<int32_t*>(S.sperm + rows);
  S.cursor = S.hist + (t.n_ann + 2);
  S.after = base + (size_t)warps * wbytes;
  return S;
}

// Resident CTAs per SM the launch bounds plan for: the single-state stages at their
// shape's count; the bilinear ones of the specialised mode counts at 2 CTAs per SM
// (80 registers, more accumulators per lane); the batched ones and the generic
// bilinear ones (16 accumulators) keep the compiler's choice (one CTA).
template <int MT, int B, int KIND, int TS>
__host__ __device__ constexpr int stage_min_blocks() {
  return (B == 1 && KIND != KIND_BIL) ? tile_shape(TS).min_blocks : ((KIND == KIND_BIL && MT > 0) ? 2 : 1);
}

template <int MT, int B, bool CPLX, int KIND, int RK, int TS>
__global__ void __launch_bounds__(32 * tile_shape(TS).warps, (stage_min_blocks<MT, B, KIND, TS>()))
    stage_df_kernel(const Tables t, const DfArgs a, const int mode) {
  constexpr bool BIL = (KIND == KIND_BIL), DOT = (KIND == KIND_DOT);
  constexpr int kWarps = tile_shape(TS).warps, kRows = tile_shape(TS).rows;
  const int M = (MT > 0) ? MT : t.M;
  // the only CTA-wide barrier: warps run independently afterwards
  const StageSmem S = stage_smem<RK>(t, M, kWarps, kRows);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row1 = a.row1;
  constexpr int kMB = (MT > 0) ? MT : 16;  // bilinear accumulators: one per mode + H_L
  dfl bil_l{0.f, 0.f};
  dfl bil_w[BIL ? kMB : 1];
#pragma unroll
  for (int q = 0; q < (BIL ? kMB : 1); ++q) bil_w[q] = dfl{0.f, 0.f};
  double dot64 = 0.0;

  for (int64_t base = a.row0 + ((int64_t)blockIdx.x * kWarps + warp) * kRows; base < row1;
       base += (int64_t)gridDim.x * kWarps * kRows)
    stage_tile<MT, B, CPLX, KIND, false, RK, kRows>(t, S.v, S.Gf, S.dtab, a, mode, base, row1, 0, S.sidx, S.socc, S.sD,
                                                    S.sOff, S.sperm, S.hist, S.cursor, bil_l, bil_w, dot64);
  if constexpr (DOT) {
    // the CTA's sum in a fixed order: lanes by shuffles, warps in turn; partial[block]
    __shared__ double red[kWarps];
    for (int o = 16; o > 0; o >>= 1) dot64 += __shfl_down_sync(0xffffffffu, dot64, o);
    if (lane == 0) red[warp] = dot64;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += red[w];
      a.partial[blockIdx.x] = sum;
    }
  }
  if constexpr (BIL) {
    // per-CTA sums of the bilinears in a fixed order: lanes by shuffles, warps in turn
    __shared__ double red[kWarps][17];
    const int nq = M + 1;
    for (int q = 0; q < nq; ++q) {
      double val = (q == 0) ? df_to(bil_l) : 0.0;
#pragma unroll
      for (int u = 0; u < kMB; ++u)
        if (q == u + 1) val = df_to(bil_w[u]);
      for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
      if (lane == 0) red[warp][q] = val;
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

constexpr int kResRows = 64;  // kets per warp tile of the resident kernel

template <int MT, bool CPLX, int RK>
__global__ void __launch_bounds__(kBlock) resident_kernel(const Tables t, const ResArgs r) {
  const int M = (MT > 0) ? MT : t.M;
  constexpr int kWarps = kBlock / 32;
  const StageSmem S = stage_smem<RK>(t, M, kWarps, kResRows);
  double2* spsi = reinterpret_cast<double2*>(S.after);
  float4* spsif = reinterpret_cast<float4*>(spsi + r.cap);
  float4* sw1 = spsif + r.cap;
  float4* sw2 = sw1 + r.cap;
  const int warp = threadIdx.x >> 5;
  dfl bil_l{0.f, 0.f}, bil_w[1] = {dfl{0.f, 0.f}};
  double dot64 = 0.0;
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
        // the sector's kets are dealt to the warps in chunks of at most kResRows,
        // evenly, so that a small sector still keeps every warp busy
        const int64_t chunk = min((int64_t)kResRows, ((int64_t)D + kWarps - 1) / kWarps);
        for (int64_t base = off + (int64_t)warp * chunk; base < off + D; base += (int64_t)kWarps * chunk)
          stage_tile<MT, 1, CPLX, KIND_STAGE, true, RK, kResRows>(t, S.v, S.Gf, S.dtab, a, d == 1 ? 1 : 0, base,
                                                             min(base + chunk, off + (int64_t)D), off, S.sidx, S.socc,
                                                             S.sD, S.sOff, S.sperm, S.hist, S.cursor, bil_l, bil_w,
                                                             dot64);
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

// ranking variant of a space
__host__ __device__ inline int rank_variant(const Tables& t) { return t.exact ? RK_EXACT : RK_PAIR; }

// shared-memory bytes of the staged table image
inline size_t stage_image_smem(const Tables& t, bool exact) {
  return (size_t)(kSmemEnd(t, exact) - kSmemFrom(t, exact) + 15) & ~(size_t)15;
}

// dynamic shared memory of a stage launch at tile shape ts
inline size_t stage_shape_smem(const Tables& t, bool exact, int ts) {
  const TileShape sh = tile_shape(ts);
  return stage_image_smem(t, exact) +
         (size_t)sh.warps * df_warp_scratch_bytes(sidx_words(t.M, exact), t.M, t.n_ann, sh.rows);
}

// The tile shape a stage launch runs at: the requested one where its shared memory
// fits a CTA on the current device (with room for the kernels' static arrays),
// otherwise the 12-warp shape (large tables, e.g. M = 16).
inline int fitting_shape(const Tables& t, bool exact, int ts) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return kWideShape;
  return stage_shape_smem(t, exact, ts) + 4096 <= (size_t)optin ? ts : kWideShape;
}

// Shared memory of the resident kernel holding `cap` kets per sector.
inline size_t resident_smem(const Tables& t, int cap) {
  return stage_image_smem(t, t.exact != 0) +
         (size_t)(kBlock / 32) * df_warp_scratch_bytes(sidx_words(t.M, t.exact != 0), t.M, t.n_ann, kResRows) +
         (size_t)cap * 64;
}

template <int MT, int RK>
int resident_launch_r(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  const size_t smem = resident_smem(t, r.cap);
  int grid = 0, rc = QB_OK;
  if (cplx) {
    auto k = resident_kernel<MT, true, RK>;
    rc = persistent_grid(k, smem, (int64_t)r.n_small * kBlock, &grid);
    if (rc) return rc;
    k<<<grid, kBlock, smem, st>>>(t, r);
  } else {
    auto k = resident_kernel<MT, false, RK>;
    rc = persistent_grid(k, smem, (int64_t)r.n_small * kBlock, &grid);
    if (rc) return rc;
    k<<<grid, kBlock, smem, st>>>(t, r);
  }
  QB_CUDA(cudaGetLastError());
  return QB_OK;
}

template <int MT>
int resident_launch_t(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  if (rank_variant(t) == RK_EXACT) return resident_launch_r<MT, RK_EXACT>(t, r, cplx, st);
  return resident_launch_r<MT, RK_PAIR>(t, r, cplx, st);
}

// Launches one stage for mode count MT (0: any M), ranking variant RK and the
// runtime batch size / coupling type / bilinear flag; `shape` selects the tile
// shape of the single-state stage (others run shape 0).  *grid (if non-NULL)
// receives the grid size.  Exact momentum: one state at a time.
template <int MT, int RK>
int stage_launch_r(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, bool bil, int shape, cudaStream_t st,
                   int* grid_out) {
  int grid = 0, rc = QB_OK;
#define QB_STAGE_CASE(BB, CC, LL, TT)                                                                   \
  {                                                                                                     \
    auto k = stage_df_kernel<MT, BB, CC, LL, RK, TT>;                                                   \
    constexpr TileShape sh = tile_shape(TT);                                                            \
    const size_t smem = stage_shape_smem(t, RK == RK_EXACT, TT);                                        \
    rc = persistent_grid(k, smem, a.row1 - a.row0, &grid, 32 * sh.warps);                               \
    if (rc) return rc;                                                                                  \
    k<<<grid, 32 * sh.warps, smem, st>>>(t, a, mode);                                                   \
  }
  if (mode < 0 || mode > 4) return fail(QB_EINTERNAL, "bad stage mode");
  // the launches of a fixed shape 0 drop to the 12-warp shape when shape 0 does not fit
  const bool wide0 = fitting_shape(t, RK == RK_EXACT, 0) != 0;
  shape = fitting_shape(t, RK == RK_EXACT, shape);
  if (mode == 4) {  // <x|H|x>
    if (B != 1) return fail(QB_EUNSUPPORTED, "the <x|H|x> reduction runs one state at a time");
    if (cplx) {
      if (wide0)
        QB_STAGE_CASE(1, true, KIND_DOT, kWideShape)
      else
        QB_STAGE_CASE(1, true, KIND_DOT, 0)
    } else {
      if (wide0)
        QB_STAGE_CASE(1, false, KIND_DOT, kWideShape)
      else
        QB_STAGE_CASE(1, false, KIND_DOT, 0)
    }
  } else if (bil) {
    if (B != 1) return fail(QB_EUNSUPPORTED, "bilinear stages run one state at a time");
    if (cplx)
      QB_STAGE_CASE(1, true, KIND_BIL, kWideShape)
    else
      QB_STAGE_CASE(1, false, KIND_BIL, kWideShape)
  } else if (cplx) {
    if (B != 1) return fail(QB_EUNSUPPORTED, "batched sweeps need a real coupling");
    if (wide0)
      QB_STAGE_CASE(1, true, KIND_STAGE, kWideShape)
    else
      QB_STAGE_CASE(1, true, KIND_STAGE, 0)
  } else {
    if constexpr (RK == RK_EXACT) {
      if (B != 1) return fail(QB_EUNSUPPORTED, "exact momentum: batched sweeps are not built");
      // the widest of 32, 24 and 12 warps that fits beside the compact ranking table
      if (!wide0)
        QB_STAGE_CASE(1, false, KIND_STAGE, 0)
      else if (fitting_shape(t, true, 2) == 2)
        QB_STAGE_CASE(1, false, KIND_STAGE, 2)
      else
        QB_STAGE_CASE(1, false, KIND_STAGE, kWideShape)
    } else {
      switch (B) {
        case 1:
          switch (shape) {
            case 1: QB_STAGE_CASE(1, false, KIND_STAGE, 1) break;
            case 2: QB_STAGE_CASE(1, false, KIND_STAGE, 2) break;
            case 3: QB_STAGE_CASE(1, false, KIND_STAGE, 3) break;
            case 4: QB_STAGE_CASE(1, false, KIND_STAGE, 4) break;
            default: QB_STAGE_CASE(1, false, KIND_STAGE, 0) break;
          }
          break;
        case 2: QB_STAGE_CASE(2, false, KIND_STAGE, kWideShape) break;
        case 4: QB_STAGE_CASE(4, false, KIND_STAGE, kWideShape) break;
        case 8: QB_STAGE_CASE(8, false, KIND_STAGE, kWideShape) break;
        default: return fail(QB_EINVAL, "batch must be 1, 2, 4 or 8");
      }
    }
  }
#undef QB_STAGE_CASE
  QB_CUDA(cudaGetLastError());
  if (grid_out) *grid_out = grid;
  return QB_OK;
}

template <int MT>
int stage_launch_t(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, bool bil, int shape, cudaStream_t st,
                   int* grid_out) {
  if (rank_variant(t) == RK_EXACT) return stage_launch_r<MT, RK_EXACT>(t, a, mode, B, cplx, bil, shape, st, grid_out);
  return stage_launch_r<MT, RK_PAIR>(t, a, mode, B, cplx, bil, shape, st, grid_out);
}

// one explicit specialisation per translation unit (qb_stage_m*.cu)
int stage_launch_m5(const Tables&, const DfArgs&, int, int, bool, bool, int, cudaStream_t, int*);
int stage_launch_m7(const Tables&, const DfArgs&, int, int, bool, bool, int, cudaStream_t, int*);
int stage_launch_m9(const Tables&, const DfArgs&, int, int, bool, bool, int, cudaStream_t, int*);
int stage_launch_m11(const Tables&, const DfArgs&, int, int, bool, bool, int, cudaStream_t, int*);
int stage_launch_any(const Tables&, const DfArgs&, int, int, bool, bool, int, cudaStream_t, int*);

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

// One stage over rows [a.row0, a.row1) in the weighted basis.  bil: the bilinear
// instantiations (adjoint modes 2, 3); mode 4 is the <x|H|x> reduction (partial[block]);
// shape: tile shape of the single-state stage (0: the default).
inline int stage_launch(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, cudaStream_t st,
                        int* grid_out = nullptr, bool bil = false, int shape = 0) {
  switch (t.M) {
    case 5: return stage_launch_m5(t, a, mode, B, cplx, bil, shape, st, grid_out);
    case 7: return stage_launch_m7(t, a, mode, B, cplx, bil, shape, st, grid_out);
    case 9: return stage_launch_m9(t, a, mode, B, cplx, bil, shape, st, grid_out);
    case 11: return stage_launch_m11(t, a, mode, B, cplx, bil, shape, st, grid_out);
    default: return stage_launch_any(t, a, mode, B, cplx, bil, shape, st, grid_out);
  }
}

}  // namespace qb
