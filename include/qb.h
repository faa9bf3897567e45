/*
 * qb -- C ABI of a GB300 (sm_103a) solver for interacting bosonic momentum
 * modes on a ring, after Eberhardt, Zamora, Kopp & Abel, "On the single
 * classical field description of interacting scalar fields" (arXiv:2111.00050).
 *
 * The many-body state lives in the Fock basis, restricted to "special Hilbert
 * spaces" (sectors) of fixed particle number N and momentum P modulo M
 * (Sec. III B).  The Hamiltonian is Eq. (Ham),
 *
 *     H = sum_p w_p a_p^dag a_p + sum_{p,q,r,s} L_{pq;rs} a_p^dag a_q^dag a_r a_s,
 *
 * summed over ORDERED tuples with p + q = r + s (mod M), where L_{pq;rs} is the
 * paper's Lambda^{rs}_{pq} / 2 (upper indices are annihilated).  Mode index i
 * carries momentum label i - (M-1)/2 for odd M and i for even M.
 *
 * Conventions shared by every call:
 *  - Complex numbers are interleaved (re, im) doubles; a state vector is a
 *    contiguous complex128 array over all sectors of a space, concatenated in
 *    the order qb_space_sectors() reports (N ascending, then P ascending).
 *    Within a sector kets are in lexicographic order of (n_0, n_1, ...).
 *  - Pointers named d_* are DEVICE pointers owned by the caller (e.g. torch
 *    tensors).  They must be 16-byte aligned, on the current CUDA device, and
 *    stay valid until the stream has finished the call's work.  The library
 *    never frees them.  Other pointers are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls that return host results synchronise on the stream before returning.
 *  - Every call returns a status: QB_OK or one of the QB_E* codes below.  On
 *    error, qb_last_error() gives a message (thread-local) and no output is
 *    written unless stated otherwise.
 */
#ifndef QB_H
#define QB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QB_OK 0
#define QB_EINVAL 1       /* bad argument: size, alignment, range, non-Hermitian or non-conserving L */
#define QB_ENOMEM 2       /* a device or host allocation failed */
#define QB_ECUDA 3        /* a CUDA runtime call or kernel launch failed */
#define QB_ETIMEOUT 4     /* a bounded device-side wait ran out */
#define QB_EINTERNAL 5    /* a device-side consistency check failed (rank out of range, ...) */
#define QB_EUNSUPPORTED 6 /* outside the compiled limits (M > QB_MAX_MODES, packed occupation > 64 bits) */

#define QB_MAX_MODES 16
#define QB_TILE_SHAPES 5  /* compiled tile shapes of the RK4 stage kernel (qb_space_set_tile_shape) */

/* Losses of qb_adjoint. */
#define QB_LOSS_Q 0  /* Q at t_f (Eq. Qparam) */
#define QB_LOSS_PO 1 /* principal eigenvalue lam_p of M_ij = <a_i^dag a_j> at t_f (Eq. POcriterion) */

/* Breaktime flags (qb_breaktime). */
#define QB_CROSSED 0
#define QB_AT_START 1
#define QB_NOT_CROSSED 2

typedef struct qb_space qb_space; /* opaque; created by qb_sector_build, freed by qb_space_free */

/* Model of Eq. (Ham).  w: [M] host doubles.  L: [M^4] host complex values as
 * (re, im) pairs, index ((p*M + q)*M + r)*M + s.  Entries on tuples that do
 * not conserve momentum must be zero (the Kronecker delta of Eq. Lambda):
 * momentum mod M when exact_momentum is 0, the plain sum of the labels
 * (Sec. III B) when exact_momentum is 1.  The library uses only the part
 * symmetric under p<->q and r<->s and requires the Hermiticity
 * L_{pq;rs} = conj(L_{rs;pq}) of that part. */
typedef struct {
  int M;
  const double* w;
  const double* L;
  int exact_momentum; /* 0: P is conserved mod M (umklapp terms allowed); 1: exactly */
} qb_model;

/* Observables of Sec. II C-E for one state, normalised by <psi|psi>.
 * Arrays are sized for QB_MAX_MODES; only the first M (or M*M, row-major)
 * entries are meaningful.  Complex entries are (re, im) pairs. */
typedef struct {
  double t;                                  /* time of the sample (set by qb_evolve_observe) */
  double norm;                               /* <psi|psi> */
  double N;                                  /* <N> */
  double H;                                  /* <H> */
  double n_tot;                              /* Tr M = sum_i <a_i^dag a_i> */
  double Q;                                  /* Eq. (Qparam): sum_j <da_j^dag da_j> / n_tot */
  double lam_p;                              /* principal eigenvalue of M (Eq. POcriterion) */
  double PO;                                 /* 1 - lam_p / n_tot */
  double gap;                                /* lam_p minus the second eigenvalue */
  double Vminus_p;                           /* Eq. (generalVminus) for a^p = sum_k xi_k a_k (Eq. a_op) */
  double a[2 * QB_MAX_MODES];                /* <a_i> */
  double Mij[2 * QB_MAX_MODES * QB_MAX_MODES]; /* <a_i^dag a_j> */
  double aa[2 * QB_MAX_MODES * QB_MAX_MODES];  /* <a_i a_j> */
  double xi[2 * QB_MAX_MODES];               /* principal eigenvector of M (unit norm, phase arbitrary) */
  double eig[QB_MAX_MODES];                  /* eigenvalues of M, ascending */
  double Vminus[QB_MAX_MODES];               /* Eq. (generalVminus) for each a_i */
} qb_obs;

/* Thread-local message for the last failing call on this thread. */
const char* qb_last_error(void);

/* ---- sectors (Sec. III B "special Hilbert spaces", App. A) -------------- */

/* Builds the space of all non-empty sectors (N, P) with n_min <= N <= n_max and
 * P in p_list[0..n_p), or every P when p_list is NULL.  P is the total
 * momentum label sum_i p_i n_i: taken mod M, in [0, M), for a model with
 * exact_momentum = 0, the exact (possibly negative) sum otherwise; sectors come
 * in the order N ascending, then P ascending.  Copies and validates the model (conservation,
 * Hermiticity), builds the combinatorial ranking tables and uploads them to the
 * current device, with two per-ket tables the space owns: the diagonal of H
 * (16 B per ket) and the occupation vector packed into 64 bits (8 B per ket),
 * plus a double-float copy of an observed state (16 B per ket).
 * Limits: 1 <= M <= QB_MAX_MODES; M * bits(n_max) <= 64; n_max <= 250;
 * the largest ket weight sqrt(n_max! / prod_m n_m!) over occupations of n_max
 * particles at most 2^160 (the RK4 stages hold psi / w(n) as fp32 pairs, with the
 * weights of each N centred on 1 by a power of two; e.g. n_max <= 206 for M = 3,
 * n_max <= 143 for M = 5); every sector dimension < 2^31; with exact momentum
 * (M-1) n_max + 1 <= 6553 (the term shifts are 16-bit), and batched sweeps
 * (batch > 1) are not built.
 * Errors: QB_EINVAL for a bad model or range, QB_EUNSUPPORTED beyond the limits,
 * QB_ECUDA / QB_ENOMEM from the device set-up.  *out receives the new space. */
int qb_sector_build(const qb_model* model, int n_min, int n_max, const int* p_list, int n_p, qb_space** out);

void qb_space_free(qb_space* space);

/* total_states: length of a state vector; n_sectors: number of sectors;
 * max_dim: largest sector dimension.  Any pointer may be NULL. */
int qb_space_info(const qb_space* space, int64_t* total_states, int* n_sectors, int64_t* max_dim);

/* Per-sector N, P label (mod M, in [0, M)), dimension and offset into the
 * state vector; each array has n_sectors entries (host).  Any may be NULL. */
int qb_space_sectors(const qb_space* space, int* N, int* P, int64_t* dim, int64_t* offset);

/* Writes the occupation vectors of global kets [first, first + count) to
 * d_occ, int32 [count][M] (device), by unranking on the GPU. */
int qb_space_basis(const qb_space* space, int64_t first, int64_t count, int* d_occ, void* stream);

/* Global index of each occupation vector d_occ[count][M] (device, int32), or
 * -1 if it is not a ket of the space; written to d_index[count] (device). */
int qb_space_rank(const qb_space* space, const int* d_occ, int64_t count, int64_t* d_index, void* stream);

/* Exact number of distinct nonzero matrix elements of H (diagonal included)
 * over all rows of the space: the work of one H psi.  Also returns the number
 * of ordered (p,q,r,s) tuples acting nontrivially, if `tuples` is not NULL. */
int qb_space_terms(const qb_space* space, int64_t* terms, int64_t* tuples, void* stream);

/* ---- initial states (Sec. II B; Sec. III B weights w^j_k(0)) ------------ */

/* |{n}> for the host occupation vector occ[M] (Eq. numEigenstate). */
int qb_init_number(qb_space* space, const int* occ, void* d_psi, void* stream);

/* Coherent state (Eq. coherentStates) with host amplitudes z[2M], restricted to
 * the space and renormalised to 1; *kept_norm (host, may be NULL) receives the
 * squared norm the space held before renormalising. */
int qb_init_coherent(qb_space* space, const double* z, void* d_psi, double* kept_norm, void* stream);

/* Field number state (Eq. fieldNumState) of n_tot particles: on kets with
 * sum n = n_tot, sqrt(n_tot!) prod_i zeta_i^{n_i} / sqrt(n_i!) with
 * zeta = z / |z|, zero elsewhere (normalised by the multinomial theorem). */
int qb_init_field_number(qb_space* space, const double* z, int n_tot, void* d_psi, void* stream);

/* ---- time evolution (Eq. Schr; the per-sector parallel scheme of Sec. III B) */

/* Bytes of device workspace qb_evolve / qb_evolve_batch need for `batch`
 * state vectors. */
int64_t qb_workspace_bytes(const qb_space* space, int batch);

/* out = H psi for one state vector (d_out and d_psi distinct, device). */
int qb_hpsi(qb_space* space, const void* d_psi, void* d_out, void* stream);

/* `steps` RK4 steps of size dt of d psi/dt = -i H psi, in place on d_psi.
 * RK4 is applied in the Horner form psi <- psi + z(psi + z/2(psi + z/3(psi +
 * z/4 psi))), z = -i dt H, which equals the classic four-stage scheme for a
 * linear time-independent H.  d_work: qb_workspace_bytes(space, 1) bytes. */
int qb_evolve(qb_space* space, void* d_psi, double dt, int64_t steps, void* d_work, void* stream);

/* Batched sweep: `batch` state vectors d_psi[batch][total], member b evolving
 * under H_b = H_w + scale[b] * H_L (one-body part unchanged, two-body part
 * scaled).  All sectors of all members advance in one launch per RK4 stage.
 * scale: host [batch].  d_work: qb_workspace_bytes(space, batch) bytes. */
int qb_evolve_batch(qb_space* space, void* d_psi, int batch, const double* scale, double dt, int64_t steps,
                    void* d_work, void* stream);

/* Execution tuning of qb_evolve for one state vector.  Leading sectors (in the
 * order of qb_space_sectors) of at most resident_max_kets kets run
 * shared-memory resident: each CTA takes such sectors from a work list and
 * advances them through every step of the call in one launch, on a side stream
 * beside the stage-by-stage launches of the larger sectors (which are captured
 * into CUDA graphs in chunks of 32 steps).  0 disables the resident path; the
 * default is 1024; values above what shared memory holds are clipped.  Results
 * do not depend on the setting: every ket goes through the same arithmetic. */
int qb_space_set_resident_max(qb_space* space, int resident_max_kets);

/* Execution tuning of the RK4 stages of qb_evolve, qb_evolve_plain and
 * qb_evolve_observe for one state vector (the per-sector parallel scheme of
 * Sec. III B, mapped onto thread blocks): the tile shape of the stage kernel, one of
 * QB_TILE_SHAPES compiled shapes given as (warps per thread block, kets per warp
 * tile, thread blocks per SM the register budget is planned for):
 *   0 (32, 64, 1) the default;  1 (16, 64, 2);  2 (24, 64, 1);  3 (12, 64, 3);
 *   4 (32, 128, 1).
 * A shape whose shared memory (the coupling tables plus the warps' tiles) does not
 * fit a thread block on the device runs as shape 3 (large tables, e.g. M = 16).
 * Every ket sums its terms in the same order under every shape, so results are
 * bit-identical; only the time differs (the Python binding's Space.autotune times
 * them on the caller's workload).  QB_EINVAL outside [0, QB_TILE_SHAPES). */
int qb_space_set_tile_shape(qb_space* space, int shape);

/* Order K of the time step of qb_evolve, qb_evolve_batch, qb_evolve_plain and
 * qb_evolve_observe: psi <- sum_{k=0..K} (z H)^k / k! psi, z = -i dt, applied in
 * the Horner form psi + z(psi + z/2(psi + ... + z/K psi)), K launches per step.
 * K = 4 (the default) is RK4; K = 2 is the second-order Taylor step of Sec. III B
 * (Eq. Q_int with the 1/2 of the second-order term).  Accepts 2, 3 or 4;
 * QB_EINVAL otherwise.  qb_adjoint requires 4 (QB_EUNSUPPORTED otherwise). */
int qb_space_set_order(qb_space* space, int order);

/* The same RK4 evolution as qb_evolve with one kernel launch per sector per
 * stage instead of one per stage for every sector: the per-sector scheme of
 * Sec. III B taken literally, kept as the comparison baseline of the batched
 * path.  Same arguments, workspace and results as qb_evolve. */
int qb_evolve_plain(qb_space* space, void* d_psi, double dt, int64_t steps, void* d_work, void* stream);

/* ---- observables (Sec. II C-E) ------------------------------------------- */

/* All observables of one state; out (host) is written after the stream syncs.
 * Every sum over kets is accumulated in FP64: the norm, <N> and <n_i> directly
 * from the FP64 state; the moments that move a ket (<a_i>, <a_i^dag a_j>,
 * <a_i a_j>) as double-float products (about 48 significant bits) of the state and
 * its weighted double-float copy, summed in double-float over 32 kets at a time and
 * added in FP64; <H> from the weighted double-float H psi, each row's contribution
 * formed and summed in FP64, with every off-diagonal term of H taken once together
 * with its Hermitian reverse (half the terms of an H psi).  The space's weighted-copy buffer (16 B per ket) is
 * overwritten.  Relative errors are of order 1e-14. */
int qb_observables(qb_space* space, const void* d_psi, qb_obs* out, void* stream);

/* Evolution with observation: series[0] is the initial state, series[k] the
 * state after k * obs_every steps, for k = 0 .. steps / obs_every (host array of
 * steps / obs_every + 1 entries; series[k].t = k * obs_every * dt). */
int qb_evolve_observe(qb_space* space, void* d_psi, double dt, int64_t steps, int obs_every, qb_obs* series,
                      void* d_work, void* stream);

/* Allocation-free variant of qb_observables (the paper has no counterpart).
 * For callers that must not allocate device memory while they run -- a
 * service under a fixed memory budget, a custom allocator that forbids
 * cudaMalloc / cudaFree after start-up, a thread that must not enter the
 * allocator because it can synchronise the device.  It writes the same
 * observables as qb_observables, but keeps its reduction partials in one
 * file-scope device array of 131072 doubles (1 MiB) that every GPU loading the
 * library holds until the process exits, and calls no allocating routine.
 * The array is shared by all calls and keeps the last call's contents; its
 * status word is cleared at the start of each call.  Calls that overlap on the
 * GPU (several streams or host threads at once) race on it: serialise them.
 * The first call on a device looks up the array's address on that device, so
 * make it before any stream capture, with that device current; the address is
 * kept for the process, which assumes one CUDA context per device for its life
 * (after cudaDeviceReset the library must be reloaded).  The grid of the
 * reduction is capped so that (4 + 2M + 4M^2 + 2) * grid + ~10 doubles fit;
 * QB_EUNSUPPORTED if even 32 CTAs would not (not reachable for M <= 16).
 * Same arguments, errors and synchronisation as qb_observables. */
int qb_observables_noalloc(qb_space* space, const void* d_psi, qb_obs* out, void* stream);

/* ---- adjoint gradients ---------------------------------------------------- */

/* Bytes of device workspace qb_adjoint needs (256-byte aligned buffer): the
 * checkpoints, steps / ckpt_every + 1 state vectors (ckpt_every = 0: one state
 * vector plus the tape, 4 * steps state-sized double-float vectors), plus 12
 * state-sized buffers and small reduction areas.  -1 for a NULL space, steps < 1
 * or ckpt_every < 0. */
int64_t qb_adjoint_workspace_bytes(const qb_space* space, int64_t steps, int ckpt_every);

/* Loss and gradients of a run from a coherent state.  The run: psi_0 = the
 * coherent state of z[2M] (Eq. coherentStates) restricted to the space and
 * renormalised; `steps` Horner RK4 steps of size dt under H = H_w + scale * H_L
 * (the space's one-body part plus `scale` times its two-body part); the loss is
 * Q (QB_LOSS_Q) or lam_p (QB_LOSS_PO) of the final state.  Outputs (host):
 * *loss; *grad_scale = d loss / d scale; grad_w[M] = d loss / d w_p;
 * grad_z[2M] = (d loss / d Re z_k, d loss / d Im z_k).  The gradient is the
 * exact discrete adjoint of the RK4 map, run backwards with the costate;
 * forward states are rebuilt by time reversal, psi_n ~ RK4 step of size -dt from
 * psi_{n+1}, restarted from a stored checkpoint every ckpt_every steps
 * (ckpt_every = 1 stores every state and reverses nothing).  ckpt_every = 0 is the
 * tape mode: the forward pass keeps each step's weighted state and its three
 * Horner stage vectors (64 bytes per ket and step), so that the backward pass runs
 * only the four costate stages per step (no reversal, no recomputed stage vectors);
 * its results equal those of ckpt_every = 1.  d_work:
 * qb_adjoint_workspace_bytes(space, steps, ckpt_every) bytes, 256-byte aligned. */
int qb_adjoint(qb_space* space, const double* z, double scale, double dt, int64_t steps, int ckpt_every,
               int loss_kind, double* loss, double* grad_scale, double* grad_w, double* grad_z, void* d_work,
               void* stream);

/* qb_adjoint plus the gradient with respect to every coupling entry (Eq. Ham):
 * grad_L[2 M^4] (host), for each ordered (p, q, r, s) the pair
 * (d loss / d Re L_{pq;rs}, d loss / d Im L_{pq;rs}) of the couplings of H, i.e.
 * scale times the space's L, each entry varied on its own in
 * H = sum_{pqrs} L_{pq;rs} a_p^dag a_q^dag a_r a_s (orderings of the two pairs are the
 * same operator and get the same value; zero off momentum conservation).  The
 * derivative along a coupling direction D is sum Re(conj(g) D) with g = grad_L[2k] +
 * i grad_L[2k + 1]; along the space's own L it equals grad_scale.  The costate
 * stages add one sweep each that forms <forward stage vector, O costate> for every
 * momentum-conserving two-body operator O.  Other arguments, results and errors as
 * qb_adjoint; QB_EINVAL if grad_L is NULL. */
int qb_adjoint_couplings(qb_space* space, const double* z, double scale, double dt, int64_t steps, int ckpt_every,
                 int loss_kind, double* loss, double* grad_scale, double* grad_w, double* grad_z, double* grad_L,
                 void* d_work, void* stream);

/* ---- breaktime and mean field (Sec. III A, IV C-D) ----------------------- */

/* First sample k with values[k] >= thr; t_br interpolates linearly between
 * samples k-1 and k spaced dt_obs apart.  flag: QB_CROSSED, QB_AT_START (k = 0,
 * t_br = 0) or QB_NOT_CROSSED (t_br = NaN).  Host only. */
int qb_breaktime(const double* values, int n, double dt_obs, double thr, double* t_br, int* flag);

/* ---- squeezing-time analysis (Sec. II E, Sec. IV E) ---------------------- */

/* Squeezing of a series vminus[0..n) of V_- samples spaced dt_obs apart
 * (normally Vminus_p, Eq. generalVminus for a^p).  Onset: the first sample k with
 * vminus[k] <= thr (the paper takes 0.8), *t_sqz interpolated linearly between
 * samples k-1 and k; *flag as for qb_breaktime (QB_AT_START if k = 0,
 * QB_NOT_CROSSED and NaN if never).  Maximal squeezing: the smallest sample,
 * refined by the vertex of the parabola through it and its two neighbours
 * (the sample itself at either end of the series): *v_min and *t_min.  Host only. */
int qb_squeezing(const double* vminus, int n, double dt_obs, double thr, double* t_sqz, int* flag, double* v_min,
                 double* t_min);

/* Mean interaction energy per occupation of the coherent amplitudes z[2M]
 * (Sec. II E): n_tot chi = n_tot^-1 sum_{pqrs} L_{pq;rs} z_p^* z_q^* z_r z_s with
 * n_tot = sum |z_p|^2 (real for a Hermitian coupling).  The paper's onset estimate
 * is t_sqz ~ 0.05 / |n_tot chi| and tau = |n_tot chi| t.  Host only. */
int qb_interaction_per_occupation(const qb_model* model, const double* z, double* ntot_chi);

/* Least-squares fit over runs (x[k], y[k]), k < n >= 2: kind 0, the power law
 * y = c0 x^c1 (a line in log x, log y; x, y > 0); kind 1, y = c0 + c1 log x
 * (x > 0).  Host only. */
int qb_fit(const double* x, const double* y, int n, int kind, double* c0, double* c1);

/* Classic RK4 of the mean-field equations (Eq. classicalFieldEqns):
 * da_k/dt = -i (w_k a_k + sum_{q,r,s} (L_{kq;rs} + L_{qk;rs}) a_q^* a_r a_s).
 * z0: [2M] host; traj: host [(steps/every + 1)][2M], row 0 = z0.  Host only. */
int qb_meanfield(const qb_model* model, const double* z0, double dt, int64_t steps, int every, double* traj);

#ifdef __cplusplus
}
#endif
#endif /* QB_H */
