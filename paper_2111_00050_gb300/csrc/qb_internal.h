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
  int o_ann;     // int32  [n_ann + 1]         first combo of annihilation pair a
  int o_pairidx; // uint8  [16][16]            pair index of (r <= s)
  int o_w;       // double [M]                 one-body w_p
  int o_gd;      // double [n_ann]             diagonal two-body coefficient mult_rs^2 L^sym_{rs;rs}
  int o_sqf;     // float2 [nmax+3]            sqrt(k) as a double-float pair (hi, lo)
  int o_Gf;      // float4 [n_combo]           G as double-float pairs (re.hi, re.lo, im.hi, im.lo)
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
  // packed occupation vector of every ket (written with the diagonal): n_m in bits
  // [m * occ_bits, (m + 1) * occ_bits), occ_bits the bit length of nmax
  int occ_bits;
  const uint64_t* occ;  // [total]
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
  int64_t scratch_doubles = 0;
  Tables t{};
  cudaStream_t capture_stream = nullptr;  // private stream on which RK4 chunks are captured into graphs
  cudaStream_t side_stream = nullptr;     // resident small sectors run here, beside the large ones
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int resident_max_kets = 1024;           // sectors up to this size run shared-memory resident
  int order = 4;                          // Taylor order of a time step (4: RK4)
  int device = 0;
  int grid_hpsi = 0;  // persistent grid sizes per kernel family
};

// error handling
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

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
// the same in FP64 arithmetic throughout (slower; for loss values)
int launch_moments_fp64(Space& s, const void* d_psi, double* out_host, void* stream);
int64_t workspace_bytes(const Space& s, int batch);
// psi (FP64 complex) -> double-float copy (float4 per ket)
int launch_to_df(const void* psi, void* psif, int64_t n, void* stream);
// psi [B][total] -> double-float copy in the weighted basis f = psi / w(n) (the stages' basis)
int launch_to_dfw(const Space& s, const void* psi, void* psif, int B, void* stream);
// observables of Sec. II C-E from the raw moments (host)
void derive(int M, const double* raw, qb_obs* out);
int device_setup(Space& s);

}  // namespace qb
