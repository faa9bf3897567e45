// Adjoint gradients of a loss at t_f (Q of Eq. Qparam, or the principal
// eigenvalue lam_p of M, Eq. POcriterion) with respect to the two-body coupling
// scale s (H = H_w + s H_L), the dispersion w_p and the coherent amplitudes z of
// the initial state (Eq. coherentStates, truncated and renormalised).
//
// Discrete adjoint of the Horner RK4 map psi' = psi + A v2, v2 = psi + A v3 / 2,
// v3 = psi + A v4 / 3, v4 = psi + A psi / 4 (A = -i dt H): with lam' the costate of
// psi', the costates of the stage vectors are g2 = A^dag lam', g3 = A^dag g2 / 2,
// g4 = A^dag g3 / 3, and lam = lam' + g2 + g3 + g4 + A^dag g4 / 4; each stage
// y = ... + c A x adds 2 dt c Im <ybar, dH/dtheta x> to d loss / d theta.  The four
// costate applications are the same double-float stage kernel run with
// z = +i c dt, and fuse the bilinears with the forward stage vectors.
//
// The forward states are not stored: psi_n comes back from psi_{n+1} by time
// reversal, psi_n ~ R(+i dt H) psi_{n+1} (exact up to O((dt |H|)^6) per step,
// |R(iy)|^2 = 1 - y^6/72 + ...), restarted from a stored checkpoint every
// ckpt_every steps so that the drift stays bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "qb_device.cuh"
#include "qb_stage.cuh"

namespace qb {

namespace {

struct SeedArgs {
  const double2* psi;
  double2* lam;
  float4* lamf;
  int kind;             // QB_LOSS_Q or QB_LOSS_PO
  double inv_norm;      // 1 / <psi|psi>
  double2 ca[16];       // Q: coefficient of (a_j psi)
  double2 cad[16];      // Q: coefficient of (a_j^dag psi)
  double c0, cN;        // Q: coefficients of psi and N psi
  double2 xi[16];       // PO: principal eigenvector of M
  double lamp;          // PO: principal eigenvalue
  int* status;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// value of psi at the ket reached from the row's ket by the occupation changes
// (e, dn), or 0 if that ket is not held
__device__ __forceinline__ double2 psi_at(const Tables& t, const View& v, const RowScratch& rs, const double2* psi,
                                          int N, int K, int nch, const int* e, const int* dn, int* status) {
  int dN = 0, dK = 0;
  for (int c = 0; c < nch; ++c) {
    dN += dn[c];
    dK += dn[c] * e[c];
  }
  const int Nt = N + dN;
  if (Nt < 0 || Nt > t.nmax) return make_double2(0.0, 0.0);
  const int Kt = (((K + dK) % t.Q) + t.Q) % t.Q;
  const int sid = __ldg(t.sec_of + Nt * t.Q + Kt);
  if (sid < 0) return make_double2(0.0, 0.0);
  const int64_t off = __ldg(t.sec_off + sid), D = __ldg(t.sec_off + sid + 1) - off;
  const int64_t r = rank_changed(t, v, rs, nch, e, dn, D);
  if (r < 0 || r >= D) {
    atomicOr(status, 1);
    return make_double2(0.0, 0.0);
  }
  return psi[off + r];
}

// lam = d loss / d psi^* at the final state, written in FP64 and double-float
__global__ void __launch_bounds__(kBlock) seed_kernel(const Tables t, const SeedArgs a) {
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
    const int N = __ldg(t.sec_N + sid), K = __ldg(t.sec_K + sid);
    setup_row(t, v, rs, N, K, D, g - off);
    const uint8_t* occ = rs.occ + tid;
    const double2 x = a.psi[g];
    double2 r = make_double2(0.0, 0.0);
    if (a.kind == QB_LOSS_Q) {
      const double c = a.c0 + a.cN * N;
      r = make_double2(c * x.x, c * x.y);
      for (int j = 0; j < M; ++j) {
        const int nj = occ[j * kBlock];
        int e[1] = {j}, up[1] = {1}, dnn[1] = {-1};
        // (a_j psi)_n = sqrt(n_j + 1) psi[n + e_j]
        const double2 pu = psi_at(t, v, rs, a.psi, N, K, 1, e, up, a.status);
        const double2 tu = cmul(a.ca[j], pu);
        const double su = sqrt((double)(nj + 1));
        r.x += su * tu.x;
        r.y += su * tu.y;
        if (nj >= 1) {  // (a_j^dag psi)_n = sqrt(n_j) psi[n - e_j]
          const double2 pd = psi_at(t, v, rs, a.psi, N, K, 1, e, dnn, a.status);
          const double2 td = cmul(a.cad[j], pd);
          const double sd = sqrt((double)nj);
          r.x += sd * td.x;
          r.y += sd * td.y;
        }
      }
    } else {
      double diag = -a.lamp;
      for (int i = 0; i < M; ++i) diag += (a.xi[i].x * a.xi[i].x + a.xi[i].y * a.xi[i].y) * occ[i * kBlock];
      r = make_double2(diag * x.x, diag * x.y);
      for (int i = 0; i < M; ++i) {
        const int ni = occ[i * kBlock];
        if (ni < 1) continue;
        for (int j = 0; j < M; ++j) {
          if (j == i) continue;
          // (a_i^dag a_j psi)_n = sqrt(n_i (n_j + 1)) psi[n - e_i + e_j]
          int e[2] = {i, j}, dn[2] = {-1, 1};
          const double2 p = psi_at(t, v, rs, a.psi, N, K, 2, e, dn, a.status);
          const double2 cij = cmul(cconj(a.xi[i]), a.xi[j]);
          const double2 tt = cmul(cij, p);
          const double s = sqrt((double)ni * (double)(occ[j * kBlock] + 1));
          r.x += s * tt.x;
          r.y += s * tt.y;
        }
      }
    }
    r.x *= a.inv_norm;
    r.y *= a.inv_norm;
    a.lam[g] = r;
    const double wi = ket_weight<0>(t, rs.occ + tid, kBlock).y;  // weighted copy, as the stages use
    a.lamf[g] = df_pack(df_of(r.x * wi), df_of(r.y * wi));
  }
}

// S0 = <bra, ket>, S_k = sum_n conj(bra_n) sqrt(n_k) ket[n - e_k] = <bra, a_k^dag ket>;
// per-CTA partials [grid][2 (M + 1)]
__global__ void __launch_bounds__(kBlock) mixed_kernel(const Tables t, const double2* bra, const double2* ket,
                                                        double* partial, int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_blob(t, smem);
  const View v = make_view(t, smem);
  const RowScratch rs = row_scratch(smem + blob_smem(t));
  const int tid = threadIdx.x, M = t.M;
  double acc[2 * (kMaxM + 1)];
  for (int k = 0; k < 2 * (kMaxM + 1); ++k) acc[k] = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < t.total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t g = base + tid;
    if (g >= t.total) break;
    const int sid = find_sector(t, g);
    const int64_t off = __ldg(t.sec_off + sid);
    const int64_t D = __ldg(t.sec_off + sid + 1) - off;
    const int N = __ldg(t.sec_N + sid), K = __ldg(t.sec_K + sid);
    setup_row(t, v, rs, N, K, D, g - off);
    const double2 b = cconj(bra[g]);
    const double2 s0 = cmul(b, ket[g]);
    acc[0] += s0.x;
    acc[1] += s0.y;
#pragma unroll
    for (int k = 0; k < kMaxM; ++k) {
      if (k >= M) break;
      const int nk = rs.occ[k * kBlock + tid];
      if (nk < 1) continue;
      int e[1] = {k}, dn[1] = {-1};
      const double2 p = psi_at(t, v, rs, ket, N, K, 1, e, dn, status);
      const double2 tt = cmul(b, p);
      const double sq = sqrt((double)nk);
      acc[2 * (k + 1)] += sq * tt.x;
      acc[2 * (k + 1) + 1] += sq * tt.y;
    }
  }
  __shared__ double red[kBlock / 32][2 * (kMaxM + 1)];
  const int lane = tid & 31, warp = tid >> 5, width = 2 * (M + 1);
#pragma unroll
  for (int k = 0; k < 2 * (kMaxM + 1); ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  if (tid < width) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += red[w][tid];
    partial[(size_t)blockIdx.x * width + tid] = s;
  }
}

// acc[c] += weight * sum_k partial[k][c], summed in a fixed order
__global__ void accumulate_kernel(const double* partial, int n, int width, double weight, double* acc) {
  for (int c = threadIdx.x; c < width; c += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partial[(size_t)k * width + c];
    acc[c] += weight * s;
  }
}

struct AdjointLayout {
  int64_t n;  // kets
  int64_t nck;
  double2* ckpt;  // [nck][n]
  float4* tape;   // tape mode: [steps][4][n] weighted state and stage vectors v4, v3, v2 of each step
  double2* psi;
  double2* lam;
  float4 *w1, *w2, *psif;  // contiguous: the RK4 workspace layout of launch_rk4
  float4 *v4, *v3, *v2, *g2, *g3, *g4, *lamf;
  double* partial;  // [max_grid][M + 1] or [max_grid][2 (M + 1)]
  double* acc;      // [M + 1]
  double* fin;      // [2 (M + 1)]
  int n_tb;         // two-body operators of the coupling gradient
  int* tb;          // [n_tb] a1 | a2 << 8 | c1 << 16 | c2 << 24
  double* tbacc;    // [2 n_tb] weighted sums of <forward stage vector, O costate>
  int64_t bytes;
};

// The two-body operators a_a1^dag a_a2^dag a_c1 a_c2 (a1 <= a2, c1 <= c2) that conserve
// momentum (mod Q, the tables' modulus), diagonal ones (a = c) included.
std::vector<int> two_body_ops(int M, int Q) {
  std::vector<int> ops;
  for (int a1 = 0; a1 < M; ++a1)
    for (int a2 = a1; a2 < M; ++a2)
      for (int c1 = 0; c1 < M; ++c1)
        for (int c2 = c1; c2 < M; ++c2)
          if ((a1 + a2) % Q == (c1 + c2) % Q) ops.push_back(a1 | (a2 << 8) | (c1 << 16) | (c2 << 24));
  return ops;
}

int64_t round256(int64_t x) { return (x + 255) & ~int64_t(255); }

// ckpt_every = 0: the tape mode (psi_0 plus four double-float vectors per step)
AdjointLayout adjoint_layout(const Space& s, int64_t steps, int ckpt_every, unsigned char* base) {
  AdjointLayout L{};
  L.n = s.t.total;
  L.nck = ckpt_every > 0 ? steps / ckpt_every + 1 : 1;
  const int64_t V = round256(L.n * 16);
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += round256(bytes);
    return p;
  };
  L.ckpt = reinterpret_cast<double2*>(take(V * L.nck));
  L.tape = ckpt_every > 0 ? nullptr : reinterpret_cast<float4*>(take(4 * V * steps));
  L.psi = reinterpret_cast<double2*>(take(V));
  L.lam = reinterpret_cast<double2*>(take(V));
  L.w1 = reinterpret_cast<float4*>(take(3 * L.n * 16));  // w1, w2, psif back to back
  L.w2 = L.w1 ? L.w1 + L.n : nullptr;
  L.psif = L.w2 ? L.w2 + L.n : nullptr;
  L.v4 = reinterpret_cast<float4*>(take(V));
  L.v3 = reinterpret_cast<float4*>(take(V));
  L.v2 = reinterpret_cast<float4*>(take(V));
  L.g2 = reinterpret_cast<float4*>(take(V));
  L.g3 = reinterpret_cast<float4*>(take(V));
  L.g4 = reinterpret_cast<float4*>(take(V));
  L.lamf = reinterpret_cast<float4*>(take(V));
  const int64_t max_grid = s.grid_hpsi;  // the largest persistent grid (SMs x 16)
  L.partial = reinterpret_cast<double*>(take(8 * max_grid * 2 * (kMaxM + 1)));
  L.acc = reinterpret_cast<double*>(take(8 * (kMaxM + 1)));
  L.fin = reinterpret_cast<double*>(take(8 * 2 * (kMaxM + 1)));
  L.n_tb = (int)two_body_ops(s.M, s.t.Q).size();
  L.tb = reinterpret_cast<int*>(take(4 * (int64_t)L.n_tb));
  L.tbacc = reinterpret_cast<double*>(take(16 * (int64_t)L.n_tb));
  L.bytes = off;
  return L;
}

}  // namespace

}  // namespace qb

using namespace qb;

extern "C" int64_t qb_adjoint_workspace_bytes(const qb_space* space, int64_t steps, int ckpt_every) {
  const Space* sp = reinterpret_cast<const Space*>(space);
  if (!sp || steps < 1 || ckpt_every < 0) return -1;
  return adjoint_layout(*sp, steps, ckpt_every, nullptr).bytes;
}

static int adjoint_impl(qb_space* space, const double* z, double scale, double dt, int64_t steps, int ckpt_every,
                        int loss_kind, double* loss, double* grad_scale, double* grad_w, double* grad_z,
                        double* grad_L, void* d_work, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp || !z || !loss || !grad_scale || !grad_w || !grad_z) return fail(QB_EINVAL, "NULL argument");
  if (steps < 1 || ckpt_every < 0) return fail(QB_EINVAL, "need steps >= 1 and ckpt_every >= 0");
  if (loss_kind != QB_LOSS_Q && loss_kind != QB_LOSS_PO) return fail(QB_EINVAL, "unknown loss kind");
  if (!std::isfinite(dt) || !std::isfinite(scale)) return fail(QB_EINVAL, "dt and scale must be finite");
  if (!d_work || (reinterpret_cast<uintptr_t>(d_work) & 255)) return fail(QB_EINVAL, "d_work must be 256-byte aligned");
  if (sp->order != 4) return fail(QB_EUNSUPPORTED, "the adjoint is the discrete adjoint of RK4 (order 4)");
  cudaStream_t st = (cudaStream_t)stream;
  const int M = sp->M;
  const AdjointLayout L = adjoint_layout(*sp, steps, ckpt_every, static_cast<unsigned char*>(d_work));
  const int64_t n = L.n;
  const bool cplx = sp->t.is_complex != 0;
  int* status = reinterpret_cast<int*>(sp->d_scratch);
  const double sc[1] = {scale};

  // ---- forward pass: psi_0 from z, checkpoints every ckpt_every steps
  int rc = qb_init_coherent(space, z, L.psi, nullptr, stream);
  if (rc) return rc;
  QB_CUDA(cudaMemcpyAsync(L.ckpt, L.psi, n * 16, cudaMemcpyDeviceToDevice, st));
  const float hs = (float)scale;
  // tape mode: vector k of step j (0: the weighted state psif_j, 1-3: v4, v3, v2)
  const int64_t vstride = round256(n * 16) / 16;
  auto slot = [&](int64_t j, int k) { return L.tape + (j * 4 + k) * vstride; };
  if (ckpt_every == 0) {
    // each step's Horner stages launched one by one, their vectors kept: v4, v3, v2
    // from psif_j, then the last stage updates psi and writes psif_{j+1} (the next
    // step's slot 0; the final one into the RK4 workspace)
    rc = launch_to_dfw(*sp, L.psi, slot(0, 0), 1, stream);
    if (rc) return rc;
    DfArgs f{};
    f.diag = sp->d_diag;
    f.scale[0] = make_float2(hs, (float)(scale - (double)hs));
    f.row0 = 0;
    f.row1 = n;
    f.status = status;
    f.psi = L.psi;
    for (int64_t j = 0; j < steps; ++j) {
      f.psif = slot(j, 0);
      for (int d = 4; d >= 1; --d) {
        f.vin = (d == 4) ? slot(j, 0) : slot(j, 4 - d);
        f.out = (d > 1) ? slot(j, 5 - d) : (j + 1 < steps ? slot(j + 1, 0) : L.psif);
        f.zre = dt / d;
        const float h = (float)f.zre;
        f.zf = make_float2(h, (float)(f.zre - (double)h));
        int grid = 0;
        rc = stage_launch(sp->t, f, d == 1 ? 1 : 0, 1, cplx, st, &grid, false, sp->tile_shape);
        if (rc) return rc;
      }
    }
  }
  for (int64_t done = 0; ckpt_every > 0 && done < steps;) {
    const int64_t seg = std::min<int64_t>(ckpt_every, steps - done);
    rc = launch_rk4(*sp, L.psi, 1, sc, dt, seg, L.w1, stream);
    if (rc) return rc;
    done += seg;
    if (done % ckpt_every == 0)
      QB_CUDA(cudaMemcpyAsync(L.ckpt + (done / ckpt_every) * n, L.psi, n * 16, cudaMemcpyDeviceToDevice, st));
  }

  // ---- loss and seed lam_N = d loss / d psi^*
  // the loss from the moments of qb_observables (FP64 reductions of double-float
  // products, about 1e-14 relative)
  qb_obs ob;
  {
    std::vector<double> raw(4 + 2 * M + 4 * (size_t)M * M, 0.0);
    rc = launch_moments(*sp, L.psi, raw.data(), stream);
    if (rc) return rc;
    if (!(raw[0] > 0.0)) return fail(QB_EINVAL, "the final state has zero norm");
    derive(M, raw.data(), &ob);
  }
  SeedArgs sa{};
  sa.psi = L.psi;
  sa.lam = L.lam;
  sa.lamf = L.lamf;
  sa.kind = loss_kind;
  sa.inv_norm = 1.0 / ob.norm;
  sa.status = status;
  if (loss_kind == QB_LOSS_Q) {
    *loss = ob.Q;
    double S = 0.0;
    for (int j = 0; j < M; ++j) S += ob.a[2 * j] * ob.a[2 * j] + ob.a[2 * j + 1] * ob.a[2 * j + 1];
    const double Nx = ob.n_tot;
    for (int j = 0; j < M; ++j) {
      sa.ca[j] = make_double2(-ob.a[2 * j] / Nx, ob.a[2 * j + 1] / Nx);    // -conj(A_j) / n_tot
      sa.cad[j] = make_double2(-ob.a[2 * j] / Nx, -ob.a[2 * j + 1] / Nx);  // -A_j / n_tot
    }
    sa.c0 = S / Nx;
    sa.cN = S / (Nx * Nx);
  } else {
    *loss = ob.lam_p;
    for (int j = 0; j < M; ++j) sa.xi[j] = make_double2(ob.xi[2 * j], ob.xi[2 * j + 1]);
    sa.lamp = ob.lam_p;
  }
  {
    const size_t smem = blob_smem(sp->t) + kRowScratchBytes;
    int grid = 0;
    rc = persistent_grid(seed_kernel, smem, n, &grid);
    if (rc) return rc;
    seed_kernel<<<grid, kBlock, smem, st>>>(sp->t, sa);
    QB_CUDA(cudaGetLastError());
  }
  QB_CUDA(cudaMemsetAsync(L.acc, 0, 8 * (kMaxM + 1), st));
  const std::vector<int> ops = two_body_ops(M, sp->t.Q);
  if (grad_L) {
    QB_CUDA(cudaMemcpy(L.tb, ops.data(), 4 * ops.size(), cudaMemcpyHostToDevice));
    QB_CUDA(cudaMemsetAsync(L.tbacc, 0, 16 * ops.size(), st));
  }

  // ---- backward pass
  DfArgs a{};
  a.diag = sp->d_diag;
  a.scale[0] = make_float2(hs, (float)(scale - (double)hs));
  a.row0 = 0;
  a.row1 = n;
  a.status = status;
  auto set_z = [&](double zre) {
    a.zre = zre;
    const float h = (float)zre;
    a.zf = make_float2(h, (float)(zre - (double)h));
  };
  auto run = [&](int mode, bool bil, double weight) -> int {
    int grid = 0;
    int r = stage_launch(sp->t, a, mode, 1, cplx, st, &grid, bil, 0);
    if (r) return r;
    if (bil) {
      accumulate_kernel<<<1, 32, 0, st>>>(L.partial, grid, M + 1, weight, L.acc);
      QB_CUDA(cudaGetLastError());
      // coupling gradient: <forward stage vector, O costate> for every two-body O
      if (grad_L) {
        r = launch_tb_bilinear(*sp, a.pair, a.vin, L.tb, L.n_tb, weight, L.tbacc, stream);
        if (r) return r;
      }
    }
    return QB_OK;
  };
  a.partial = L.partial;
  for (int64_t step = steps - 1; step >= 0; --step) {
    // psi_step: a checkpoint, or one RK4 step backwards in time from psi_{step+1}
    // (tape mode: the stored weighted state and stage vectors of the step)
    float4* psif = L.psif;
    float4 *v4 = L.v4, *v3 = L.v3, *v2 = L.v2;
    if (ckpt_every == 0) {
      psif = slot(step, 0);
      v4 = slot(step, 1);
      v3 = slot(step, 2);
      v2 = slot(step, 3);
    } else if (step % ckpt_every == 0) {
      QB_CUDA(cudaMemcpyAsync(L.psi, L.ckpt + (step / ckpt_every) * n, n * 16, cudaMemcpyDeviceToDevice, st));
      rc = launch_to_dfw(*sp, L.psi, L.psif, 1, stream);
      if (rc) return rc;
    } else {
      rc = launch_rk4(*sp, L.psi, 1, sc, -dt, 1, L.w1, stream);  // leaves the weighted copy in psif
      if (rc) return rc;
    }
    // forward stage vectors of this step (tape mode: stored)
    a.nbasef = 0;
    if (ckpt_every > 0) {
      a.psif = L.psif;
      a.vin = L.psif;
      a.out = L.v4;
      set_z(dt / 4);
      if ((rc = run(0, false, 0.0))) return rc;
      a.vin = L.v4;
      a.out = L.v3;
      set_z(dt / 3);
      if ((rc = run(0, false, 0.0))) return rc;
      a.vin = L.v3;
      a.out = L.v2;
      set_z(dt / 2);
      if ((rc = run(0, false, 0.0))) return rc;
    }
    // costates: g2 = A^dag lam', g3 = A^dag g2 / 2, g4 = A^dag g3 / 3, lam = lam' + g2 + g3 + g4 + A^dag g4 / 4
    a.vin = L.lamf;
    a.pair = v2;
    a.out = L.g2;
    set_z(-dt);
    if ((rc = run(2, true, 1.0))) return rc;
    a.vin = L.g2;
    a.pair = v3;
    a.out = L.g3;
    set_z(-dt / 2);
    if ((rc = run(2, true, 0.5))) return rc;
    a.vin = L.g3;
    a.pair = v4;
    a.out = L.g4;
    set_z(-dt / 3);
    if ((rc = run(2, true, 1.0 / 3.0))) return rc;
    a.vin = L.g4;
    a.pair = psif;
    a.psi = L.lam;
    a.basef[0] = L.g2;
    a.basef[1] = L.g3;
    a.basef[2] = L.g4;
    a.nbasef = 3;
    a.out = L.lamf;
    set_z(-dt / 4);
    if ((rc = run(3, true, 0.25))) return rc;
  }

  // tape mode: psi still holds the final state; psi_0 is checkpoint 0
  if (ckpt_every == 0) QB_CUDA(cudaMemcpyAsync(L.psi, L.ckpt, n * 16, cudaMemcpyDeviceToDevice, st));
  // ---- initial-state gradient: d psi_0 / d z_k through a_k^dag and the renormalisation
  double hacc[kMaxM + 1];
  QB_CUDA(cudaMemcpyAsync(hacc, L.acc, 8 * (M + 1), cudaMemcpyDeviceToHost, st));
  std::vector<double> lamps(2 * (M + 1)), psips(2 * (M + 1));
  {
    const size_t smem = blob_smem(sp->t) + kRowScratchBytes;
    int grid = 0;
    rc = persistent_grid(mixed_kernel, smem, n, &grid);
    if (rc) return rc;
    const int width = 2 * (M + 1);
    mixed_kernel<<<grid, kBlock, smem, st>>>(sp->t, L.lam, L.psi, L.partial, status);
    QB_CUDA(cudaGetLastError());
    QB_CUDA(cudaMemsetAsync(L.fin, 0, 8 * width, st));
    accumulate_kernel<<<1, 64, 0, st>>>(L.partial, grid, width, 1.0, L.fin);
    QB_CUDA(cudaMemcpyAsync(lamps.data(), L.fin, 8 * width, cudaMemcpyDeviceToHost, st));
    QB_CUDA(cudaStreamSynchronize(st));
    mixed_kernel<<<grid, kBlock, smem, st>>>(sp->t, L.psi, L.psi, L.partial, status);
    QB_CUDA(cudaGetLastError());
    QB_CUDA(cudaMemsetAsync(L.fin, 0, 8 * width, st));
    accumulate_kernel<<<1, 64, 0, st>>>(L.partial, grid, width, 1.0, L.fin);
    QB_CUDA(cudaMemcpyAsync(psips.data(), L.fin, 8 * width, cudaMemcpyDeviceToHost, st));
  }
  int hstat = 0;
  QB_CUDA(cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  if (hstat) {
    QB_CUDA(cudaMemset(status, 0, sizeof(int)));
    return fail(QB_EINTERNAL, "device-side consistency check failed (status " + std::to_string(hstat) + ")");
  }
  // each bilinear stage adds 2 dt c Im <ybar, dH x>: Im <x, H_L p> = -(stored H_L sum)
  *grad_scale = -2.0 * dt * hacc[0];
  if (grad_L) {
    // d loss / d L_{pq;rs} for H = sum L_{pq;rs} a_p^dag a_q^dag a_r a_s: the operator of
    // the entry, O_{A;C}, against the stored sums of its reverse O_{C;A} (the sweep
    // pairs the forward vector as bra with the costate as ket):
    // d/dRe L = -2 dt Im B_{C;A}, d/dIm L = 2 dt Re B_{C;A}; every ordering of the
    // two pairs is the same operator, so it gets the same value
    std::vector<double> B(2 * ops.size());
    QB_CUDA(cudaMemcpyAsync(B.data(), L.tbacc, 16 * ops.size(), cudaMemcpyDeviceToHost, st));
    QB_CUDA(cudaStreamSynchronize(st));
    const size_t M4 = (size_t)M * M * M * M;
    std::fill(grad_L, grad_L + 2 * M4, 0.0);
    auto at = [&](int p, int q, int r2, int s2) { return (((size_t)p * M + q) * M + r2) * M + s2; };
    for (size_t e = 0; e < ops.size(); ++e) {
      const int a1 = ops[e] & 0xff, a2 = (ops[e] >> 8) & 0xff, c1 = (ops[e] >> 16) & 0xff, c2 = (ops[e] >> 24) & 0xff;
      const int rev = c1 | (c2 << 8) | (a1 << 16) | (a2 << 24);
      const size_t er = (size_t)(std::find(ops.begin(), ops.end(), rev) - ops.begin());
      if (er >= ops.size()) return fail(QB_EINTERNAL, "two-body operator without its reverse");
      const double gre = -2.0 * dt * B[2 * er + 1], gim = 2.0 * dt * B[2 * er];
      const int P[2][2] = {{a1, a2}, {a2, a1}}, R[2][2] = {{c1, c2}, {c2, c1}};
      for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
          const size_t ix = at(P[u][0], P[u][1], R[v][0], R[v][1]);
          grad_L[2 * ix] = gre;
          grad_L[2 * ix + 1] = gim;
        }
    }
  }
  for (int q = 0; q < M; ++q) grad_w[q] = 2.0 * dt * hacc[q + 1];
  const double cre = lamps[0];  // Re <lam_0, psi_0>
  for (int k = 0; k < M; ++k) {
    const double Gr = lamps[2 * (k + 1)], Gi = lamps[2 * (k + 1) + 1];
    const double Hr = psips[2 * (k + 1)], Hi = psips[2 * (k + 1) + 1];
    grad_z[2 * k] = 2.0 * Gr - 2.0 * cre * Hr;
    grad_z[2 * k + 1] = -2.0 * Gi + 2.0 * cre * Hi;
  }
  return QB_OK;
}

extern "C" int qb_adjoint(qb_space* space, const double* z, double scale, double dt, int64_t steps, int ckpt_every,
                          int loss_kind, double* loss, double* grad_scale, double* grad_w, double* grad_z,
                          void* d_work, void* stream) {
  return adjoint_impl(space, z, scale, dt, steps, ckpt_every, loss_kind, loss, grad_scale, grad_w, grad_z, nullptr,
                      d_work, stream);
}

extern "C" int qb_adjoint_couplings(qb_space* space, const double* z, double scale, double dt, int64_t steps, int ckpt_every,
                            int loss_kind, double* loss, double* grad_scale, double* grad_w, double* grad_z,
                            double* grad_L, void* d_work, void* stream) {
  if (!grad_L) return fail(QB_EINVAL, "grad_L must be non-NULL");
  return adjoint_impl(space, z, scale, dt, steps, ckpt_every, loss_kind, loss, grad_scale, grad_w, grad_z, grad_L,
                      d_work, stream);
}
