// Internal structures shared by the host code (qb_host.cpp) and the CUDA
// kernels (qb_kernels.cu).  Not part of the public ABI (include/qb.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qb.h"

namespace qb {

// Shifts of a suffix-state index are stored as unsigned bytes offset by this bias
// (a shift lies in [-4M, 5M) for M <= 16).
constexpr int kDeltaBias = 64;

// Everything a kernel needs to walk one space, passed by value.
//
// Ranking of a ket n within its sector (N, K), K = sum_i i n_i mod M (mode
// index momentum), in lexicographic order (n_0 most significant):
//   rank(n) = D - 1 - sum_{m=1}^{M-1} E_m(rem_m, krem_m),
//   rem_m = sum_{i>=m} n_i,  krem_m = sum_{i>=m} i n_i mod M,
//   E_m(rem, k) = cnt[m-1][rem-1][(k - (m-1)) mod M]  (0 for rem < 1),
// where cnt[m][n][k] counts the fillings of modes m..M-1 with n particles and
// index momentum k.  E is stored as E[m][rem + 2][kk] for kk in [0, 2M) with
// E[..][kk] = E_m(rem, kk mod M), so that shifting (rem, krem) by a term's
// (dc, dk mod M) is one integer add on the flat index:
//   idx(m, rem, krem) = (m * rem_w + rem + 2) * 2M + krem.
struct Tables {
  int M;
  int Q;         // momentum modulus of the tables: M (mod-M conservation) or (M-1) nmax + 1 (exact)
  int exact;     // 1: momentum conserved exactly (Q exceeds every momentum sum)
  int sm_from;   // first byte of the image the row kernels stage in shared memory (cnt, E stay global below it)
  int nmax;      // largest N of the space
  int rem_w;     // nmax + 5
  int n_ann;     // M(M+1)/2 unordered annihilation pairs (r <= s)
  int n_combo;   // (annihilation pair, creation pair) combinations, zero couplings included
  int is_complex;
  int blob_bytes;  // size of the shared-memory image
  // byte offsets of the sub-tables inside the image
  int o_cnt;     // uint32 [(M+1)][nmax+1][Q]
  int o_E;       // int32  [M][rem_w][2Q]
  int o_sqrt;    // double [nmax+3]            sqrt(k)
  int o_pq;      // uint32 [n_combo]           p | q<<8 | lo<<16 | hi<<24
  int o_G;       // double [n_combo][2]        conj(mult * L^sym_{pq;rs}) (re, im)
  int o_delta;   // uint8  [n_combo][16]       kDeltaBias + flat-index shift of the suffix state at mode m
                 //   (exact: int16 [n_combo][16], the shift itself)
  int o_Ex;      // exact momentum, when it fits a CTA: the compact ranking table, mode m (1 .. M-1)
                 //   at byte ex_base[m], int32 [rem_w][ex_w[m]], column skr - m rem (the suffix
                 //   momentum of mode m lies in [m rem, (M-1) rem]); empty otherwise (o_Ex = o_ann)
  int ex_smem;   // 1: the stage kernels rank exact-momentum targets in the compact table
  int ex_w[16];
  int ex_base[16];
  int o_dex;     // int16  [n_combo][16]       shifts of the flat compact index per mode (exact, compact)
  int o_ann;     // int32  [n_ann + 1]         first combo of annihilation pair a
  int o_hs;      // int32  [n_ann]             first combo of pair a whose creation pair (p, q) has a
                 //   larger pair index: <x|H|x> takes each term once with its reverse
  int o_pairidx; // uint8  [16][16]            pair index of (r <= s)
  int o_w;       // double [M]                 one-body w_p
  int o_gd;      // double [n_ann]             diagonal two-body coefficient mult_rs^2 L^sym_{rs;rs}
  int o_sqf;     // float2 [nmax+3]            sqrt(k) as a double-float pair (hi, lo)
  // The stage kernel's per-term tables are column arrays of ncp entries (n_combo
  // rounded up to a multiple of 4), so that the 32 lanes of a warp, each on its own
  // term, load 8 or 4 bytes apiece from densely packed rows:
  int ncp;
  int o_Gf;      // float2 [2][ncp]            G as double-float pairs: [0][j] (re.hi, re.lo), [1][j] (im.hi, im.lo)
  int o_dsw;     // uint2 [ncp], then uint32 [nsw - 2][ncp]: byte shifts of the suffix index, two modes
                 //   per word (nsw = max(1, M / 2) words): word k holds 4 shift(2k+1) + 65536 * 4
                 //   shift(2k+2) (the ranking table's byte offsets of modes 2k+1 and 2k+2 added in one
                 //   32-bit add, see the stage kernel); words 0 and 1 side by side, the rest one array
                 //   per word
  int sw_ok;     // 1: every byte offset into the ranking table fits 16 bits (required for mod-M momentum)
  const unsigned char* blob;  // device pointer to the image
  // sectors
  int n_sectors;
  const int64_t* sec_off;  // [n_sectors + 1]
  const int32_t* sec_N;    // [n_sectors]
  const int32_t* sec_K;    // [n_sectors] index momentum
  const int32_t* sec_of;   // [(nmax + 1) * Q] sector id of (N, K) or -1
  int64_t total;
  // ket weights w(n) = sqrt(N! / prod_m n_m!) = prod_m sqrt(C(rem_m, n_m)), rem_m the
  // particles in modes m..M-1: entry [rem * (nmax + 1) + k] = (sqrt(C(rem, k)), its inverse)
  const double2* wtab;
  // per particle number N: (2^-e_N, 2^e_N), e_N = round(log2(w_max(N)) / 2) with w_max(N)
  // the largest ket weight of N particles in M modes; the stages use w(n) 2^-e_N, which
  // keeps every weight of the sector within [2^-k, 2^k], k = log2(w_max) / 2 + 1/2.  A
  // constant per sector is a similarity inside each diagonal block of H, so the
  // weighted operator is unchanged; a power of two changes no rounding.
  const double2* wscale;
  // packed occupation vector of every ket (written with the diagonal): n_m in bits
  // [m * occ_bits, (m + 1) * occ_bits), occ_bits the bit length of nmax
  int occ_bits;
  const uint64_t* occ;  // [total]
  const double* wi;     // [total] 1 / w(n) of every ket (the centred ket weight; ket_weight)
};

struct Space {
  int M = 0;
  int Q = 0;       // momentum modulus (Tables::Q)
  int exact = 0;   // momentum conserved exactly
  int nmax = 0, nmin = 0;
  std::vector<double> w;                  // [M]
  std::vector<double> Lsym;               // [M^4][2]
  std::vector<int> secN, secP, secK;      // per sector
  std::vector<int64_t> secDim, secOff;    // secOff has n_sectors + 1 entries
  std::vector<uint64_t> cnt;              // host copy of the fill counts
  std::vector<int> secOf;                 // [(nmax+1) * Q]
  std::vector<unsigned char> blob;        // host copy of the shared-memory image
  int64_t maxDim = 0;
  // device allocations owned by the space
  unsigned char* d_blob = nullptr;
  int64_t* d_secOff = nullptr;
  int32_t* d_secN = nullptr;
  int32_t* d_secK = nullptr;
  int32_t* d_secOf = nullptr;
  double* d_scratch = nullptr;  // reduction partials
  float4* d_diag = nullptr;     // per ket: one-body and two-body diagonal as double-float pairs
  float4* d_obsf = nullptr;     // double-float copy of the state being observed (qb_observables)
  double2* d_wtab = nullptr;    // ket-weight factors (Tables::wtab)
  uint64_t* d_occ = nullptr;    // packed occupation vectors (Tables::occ)
  double* d_wi = nullptr;       // inverse ket weights (Tables::wi)
  int64_t scratch_doubles = 0;
  Tables t{};
  cudaStream_t capture_stream = nullptr;  // private stream on which RK4 chunks are captured into graphs
  cudaStream_t side_stream = nullptr;     // resident small sectors run here, beside the large ones
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int resident_max_kets = 1024;           // sectors up to this size run shared-memory resident
  int order = 4;                          // Taylor order of a time step (4: RK4)
  int tile_shape = 0;                     // tile shape of the single-state stage kernel (qb_stage.cuh)
  int device = 0;
  int grid_hpsi = 0;  // persistent grid sizes per kernel family
};

// error handling
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
// reads the space's device status word (clearing it): QB_EINTERNAL if a device-side
// check failed since the last read
int check_status(const Space& s, cudaStream_t st);

// Raw moments of one state (doubles): [0] norm, [1] <N> norm, [2] <H> norm, [3] unused,
// then <a_i> [M], <a_i^dag a_j> [M*M], <a_i a_j> [M*M] as (re, im) pairs.
__host__ __device__ inline int nmoments(int M) { return 4 + 2 * M + 4 * M * M; }
// Columns of the per-CTA partials of the observables' first pass: norm, <N>, <n_i> [M].
__host__ __device__ inline int nprep(int M) { return M + 2; }

// Scratch layout of a space (doubles), sized at set-up for the largest persistent grid
// G = SMs * 16:  [0, 2) status word | moment partials [G nmom] | moment sums [nmom] |
// bilinear / <H> partials [(M + 1) G] | their sums [QB_MAX_MODES + 2] | amplitude table
// [2 M (nmax + 1)] | initial-state norm [2] | first-pass partials [nprep G] | their sums [nprep]
inline int64_t scratch_doubles_for(int M, int nmax, int64_t G) {
  return 2 + G * nmoments(M) + nmoments(M) + (int64_t)(M + 1) * G + QB_MAX_MODES + 2 + 2 * (int64_t)M * (nmax + 1) +
         2 + G * nprep(M) + nprep(M);
}
inline int64_t max_grid_of(const Space& s) { return s.scratch_doubles > 0 ? (int64_t)s.grid_hpsi : 0; }
inline double* partial_area(const Space& s) { return s.d_scratch + 2; }
inline double* final_area(const Space& s) { return partial_area(s) + max_grid_of(s) * nmoments(s.M); }
inline double* dot_area(const Space& s) { return final_area(s) + nmoments(s.M); }
inline double* dot_final(const Space& s) { return dot_area(s) + (int64_t)(s.M + 1) * max_grid_of(s); }
inline double* table_area(const Space& s) { return dot_final(s) + QB_MAX_MODES + 2; }
inline double* init_final(const Space& s) { return table_area(s) + 2 * (size_t)s.M * (s.nmax + 1); }
inline double* prep_area(const Space& s) { return init_final(s) + 2; }
inline double* prep_final(const Space& s) { return prep_area(s) + max_grid_of(s) * nprep(s.M); }

// launchers (qb_kernels.cu); all return a QB_* status
int launch_hpsi(const Space& s, const void* d_v, void* d_out, void* stream);
int launch_rk4(Space& s, void* d_psi, int batch, const double* scale, double dt, int64_t steps, void* d_work,
               void* stream, bool plain = false);
int launch_unrank(const Space& s, int64_t first, int64_t count, int* d_occ, void* stream);
int launch_rank(const Space& s, const int* d_occ, int64_t count, int64_t* d_index, void* stream);
int launch_terms(const Space& s, int64_t* terms, int64_t* tuples, void* stream);
int launch_init_table(const Space& s, const double* table_host, int only_N, void* d_psi, double* norm2,
                      void* stream);
int launch_scale(const Space& s, void* d_psi, double factor, void* stream);
int launch_number(const Space& s, int64_t index, void* d_psi, void* stream);
// raw moments: out[0]=norm, out[1]=<N>, out[2]=<H>, then a[M], Mij[M*M], aa[M*M] complex
int launch_moments(Space& s, const void* d_psi, double* out_host, void* stream);
// d_acc[2e], d_acc[2e + 1] += weight * <bra, O_e ket> (re, im) for the two-body operators
// O_e = a_a1^dag a_a2^dag a_c1 a_c2 listed in d_tb[e] = a1 | a2 << 8 | c1 << 16 | c2 << 24;
// bra and ket are weighted double-float vectors of the space (as the stage kernels hold them)
int launch_tb_bilinear(Space& s, const float4* bra, const float4* ket, const int* d_tb, int n_tb, double weight,
                       double* d_acc, void* stream);
int64_t workspace_bytes(const Space& s, int batch);
// psi (FP64 complex) -> double-float copy (float4 per ket)
int launch_to_df(const void* psi, void* psif, int64_t n, void* stream);
// psi [B][total] -> double-float copy in the weighted basis f = psi / w(n) (the stages' basis)
int launch_to_dfw(const Space& s, const void* psi, void* psif, int B, void* stream);
// observables of Sec. II C-E from the raw moments (host)
void derive(int M, const double* raw, qb_obs* out);
// log2 of the largest ket weight sqrt(N! / prod_m n_m!) over all occupations of N
// particles in M modes (the most even one), and the largest log2 weight a space may
// reach: the stage vectors hold psi / w as fp32 pairs, so the centred weights
// w 2^-e_N must stay within 2^+-80 (qb_sector_build refuses deeper spaces)
double log2_max_ket_weight(int M, int N);
constexpr double kMaxLog2KetWeight = 160.0;
int device_setup(Space& s);

}  // namespace qb
