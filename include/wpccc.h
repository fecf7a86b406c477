/*
 * wpccc.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of the
 * wave-packet convergent-close-coupling (WP-CCC) method for ion-atom collisions
 * (Abdurakhmanov, Antonio, Cytowski, Kadyrov, "Portable GPU implementation of the
 * WP-CCC ion-atom collisions code", arXiv:2403.04252).
 *
 * The paper's most expensive part (Sec. II, Eq. 1) is the set of coupled
 * first-order equations
 *
 *     i v [[I, K], [K^+, I]] d/dz [F; G] = [[D_T, Q], [Q^+, D_P]] [F; G]
 *
 * along straight-line projectile paths (impact parameter b, speed v, position z).
 * Written as dX/dz = M X with M = -(i/v) S^{-1} H (Eq. 2-4), it is advanced by
 * classical RK4 (Algorithm 1).  In this header
 *   S = [[I, K], [K^+, I]]       overlap matrix       (paper: the matrix left of d/dz)
 *   H = [[D_T, Q], [Q^+, D_P]]   coupling matrix      (paper: the matrix on the right)
 *   X = S^{-1} H                 solution of the linear system (paper: ZGESV)
 *   c = [F; G]                   amplitudes (paper: the solution vector X of Eq. 2-3)
 *
 * Conventions shared by every call:
 *   - complex numbers are two doubles (re, im), i.e. C99 double _Complex /
 *     cuDoubleComplex / numpy complex128;
 *   - N x N matrices are column-major (LAPACK layout), element (i, j) at i + j*N;
 *     a batch of matrices is contiguous, matrix k at offset k*N*N elements;
 *   - state order is: every target state, then every projectile state, each in
 *     the order given in wpccc_centre_desc;
 *   - pointers documented "host" are read during the call only and may be freed
 *     after it returns; pointers documented "device" are owned by the caller and
 *     must stay valid until the work queued on `stream` has finished;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     calls are asynchronous with respect to the host unless stated otherwise;
 *   - every call returns a wpccc_status and never aborts; on failure
 *     wpccc_last_error() describes the cause.  A call that fails argument
 *     checking queues no GPU work.
 *
 * Atomic units throughout (hbar = m_e = e = 1).
 */
#ifndef WPCCC_H
#define WPCCC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define WPCCC_API __attribute__((visibility("default")))
#else
#define WPCCC_API
#endif

typedef enum {
    WPCCC_OK = 0,
    WPCCC_EINVAL = 1,      /* invalid argument (null pointer, size out of range, inconsistent basis) */
    WPCCC_ENOMEM = 2,      /* device or host allocation failed */
    WPCCC_ESINGULAR = 3,   /* a linear system had an exactly zero pivot (ZGESV info > 0) */
    WPCCC_ENONFINITE = 4,  /* amplitudes became NaN or infinite during propagation */
    WPCCC_ECUDA = 5,       /* a CUDA runtime call or kernel launch failed */
    WPCCC_EUNSUPPORTED = 6, /* a mode this build does not provide */
    WPCCC_ETIMEOUT = 7,    /* a bounded wait inside a kernel gave up (see wpccc_basis_set_wait_limit);
                              the kernel returned cleanly and the device stays usable */
    WPCCC_ENOCONV = 8      /* the FP64 iterative refinement of a reduced-precision form did not converge (see
                              wpccc_basis_set_refine_tolerance); the amplitudes are returned but not trusted */
} wpccc_status;

/* Largest orbital angular momentum a basis may hold, and largest system size.  Beyond about 2840 states
 * the RK4 sweep of the two-centre forms no longer fits one block's shared memory (EINVAL from
 * wpccc_propagate); one-centre bases then propagate with the vectors in global memory (see
 * wpccc_basis_set_rk4_layout). */
#define WPCCC_LMAX 10
#define WPCCC_NMAX 8192

/* Opaque handle: the basis and every z-independent table, resident on one device. */
typedef struct wpccc_basis_s* wpccc_basis;

/*
 * One centre's basis (Sec. II, first paragraph: bound eigenstates plus
 * wave-packet pseudostates).  A state is a radial function f_{nl}(r) times a
 * spherical harmonic Y_{lm} quantised along the projectile velocity.  All
 * pointers are host pointers.
 */
typedef struct {
    double Z;              /* charge of this centre's nucleus (the projectile's charge for the
                              projectile centre; in one-centre mode only P.Z is read) */
    int n_rad;             /* number of radial functions, >= 1 */
    const int* rad_l;      /* [n_rad] orbital angular momentum of each radial function, 0..WPCCC_LMAX */
    const double* f;       /* [n_rad][Nr] row-major: f_a(r_i), the radial function on the r-grid,
                              normalised so that sum_i w_i r_i^2 f_a(r_i)^2 = 1 */
    int n_states;          /* number of states on this centre */
    const int* st_rad;     /* [n_states] radial function of each state */
    const int* st_m;       /* [n_states] magnetic quantum number, |m| <= l */
    const double* st_eps;  /* [n_states] energy of each state */
} wpccc_centre_desc;

/*
 * The whole expansion basis and the quadrature rules.  Host pointers.
 * Two-centre mode requires every radial function of each centre to appear with
 * all 2l+1 values of m (the molecular-frame integrals are evaluated for q >= 0
 * and completed by the q -> -q reflection).
 */
typedef struct {
    int n_centres;         /* 1: one-centre (Eq. 5, no solve), 2: two-centre (Eq. 4) */
    int Nr;                /* r-grid points, >= 5 */
    const double* r;       /* [Nr] strictly increasing radii, r[0] > 0 (Sec. II: 0..~100 a.u.) */
    const double* w;       /* [Nr] integration weights of the grid (used for Eq. 7) */
    wpccc_centre_desc T;   /* target centre */
    wpccc_centre_desc P;   /* projectile centre (only P.Z is read when n_centres == 1) */
    int Geta;              /* Gauss-Laguerre points for eta in Eq. 9 (ignored in one-centre mode) */
    const double* s;       /* [Geta] Laguerre nodes */
    const double* ws;      /* [Geta] Laguerre weights times exp(s) */
    int Gtau;              /* Gauss-Legendre points for tau in Eq. 9 */
    const double* tau;     /* [Gtau] nodes on (-1, 1) */
    const double* wtau;    /* [Gtau] weights */
    double gamma;          /* eta = 1 + s / (gamma * R) maps the Laguerre variable onto [1, inf) */
    /* Short-range part of a one-electron (Li-like) target potential.  The paper treats bare
       nuclei; with mp_c != 0 the target potential is
         V_T(r) = -[T.Z + mp_c exp(-mp_a r) (1 + mp_b r)] / r,
       so the transfer integral Q carries V_T(r_T) in place of -T.Z/r_T and D_P gains the
       short-range part between projectile states (integrated on the Eq. 9 (eta, tau) rule; only
       equal-q pairs couple in the molecular frame).  The target's states must then be eigenstates
       of this potential.  mp_c = 0 (zero-initialised descriptors) is the bare-nucleus case. */
    double mp_c, mp_a, mp_b;
} wpccc_basis_desc;

/*
 * A set of straight-line paths.  Host pointers.  Path p has speed v[p] > 0,
 * impact parameter b[p] > 0 and n_z[p] >= 1 strictly increasing z nodes
 * z[off_p .. off_p + n_z[p] - 1] with off_p = n_z[0] + ... + n_z[p-1]; it is
 * advanced by n_z[p] - 1 RK4 steps (Algorithm 1; the paper's z-grid of Sec. II
 * or any other grid).
 */
typedef struct {
    int n_paths;
    const double* b;
    const double* v;
    const int* n_z;
    const double* z;
} wpccc_paths;

/*
 * Builds a basis on `device`.  As in Sec. II, every z- and b-independent table is
 * made once and kept in device memory for all later calls: this uploads the r-grid,
 * the radial functions, energies and quadrature rules, and computes on the GPU the
 * radial multipole table F_{n'l'nl lambda}(r_i) of Eq. 7 at every grid radius and
 * the angular coefficients of Eq. 6.  Synchronous.  On success *out owns device
 * memory until wpccc_basis_destroy.  Errors: EINVAL (inconsistent description, or a
 * non-finite value in r, w, the radial tables, energies, charges, quadrature rules or
 * model-potential parameters; checked on the host before any device work), ENOMEM, ECUDA.
 */
WPCCC_API wpccc_status wpccc_basis_create(const wpccc_basis_desc* desc, int device, wpccc_basis* out);

/* Frees everything the basis owns.  Synchronises the basis' device first.  NULL is accepted. */
WPCCC_API wpccc_status wpccc_basis_destroy(wpccc_basis basis);

/* Sizes of the basis: N_T target states, N_P projectile states (0 in one-centre mode). */
WPCCC_API wpccc_status wpccc_basis_info(wpccc_basis basis, int* N_T, int* N_P);

/*
 * Matrix elements at nz projectile positions of one path (Eq. 1, 6-9):
 *   S[k] = [[I, K], [K^+, I]],  H[k] = [[D_T, Q], [Q^+, D_P]]  at z = z[k]
 * with every element between states i and j carrying exp(i (eps_i - eps_j) z / v).
 *   D_T: Eq. 6 with the projectile charge, F of Eq. 7 interpolated at R = sqrt(b^2+z^2)
 *        by 5-point Lagrange interpolation on the r-grid;
 *   D_P: the same expansion about the projectile with the target charge at -R;
 *   K, Q: Eq. 9 on the (eta, tau) rule with the ETF phase exp(i v z eta tau / 2)
 *        and J_{q-q'}, rotated to the collision frame by Eq. 8; Q carries -Z_T/r_T
 *        (V_T(r_T) for a model-potential target, see wpccc_basis_desc);
 *        the lower-left block of H is Q^+, as Eq. 1 prints it (H Hermitian).
 * In one-centre mode S[k] = I and H[k] = D_T.
 *   z      host   [nz] positions
 *   S, H   device [nz][N][N] complex128, column-major; fully overwritten
 * Errors: EINVAL (nz < 1, b <= 0, v <= 0, null pointers), ENOMEM, ECUDA.
 */
WPCCC_API wpccc_status wpccc_matrix_elements(wpccc_basis basis, double b, double v, int nz, const double* z,
                                   void* S, void* H, void* stream);

/*
 * wpccc_matrix_elements with the element arithmetic of a reduced-precision form, to measure its element
 * error against the FP64 elements (the paper has no counterpart):
 *   precision_mode 0 FP64 (= wpccc_matrix_elements), 1 the Eq. 9 contraction on the FP32 pipe,
 *   3 the Eq. 9 contraction on the tensor cores with four slices, 4 the same to FP64 accuracy (see
 *   wpccc_propagate).  S and H are returned in FP64.
 * Errors: as wpccc_matrix_elements; EUNSUPPORTED for other modes, one-centre bases or model-potential
 * targets in modes 1, 3 and 4.
 */
WPCCC_API wpccc_status wpccc_matrix_elements_precision(wpccc_basis basis, double b, double v, int nz,
                                                       const double* z, void* S, void* H, int precision_mode,
                                                       void* stream);

/*
 * wpccc_matrix_elements without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot let the library allocate device
 * memory inside a call, e.g. a host framework that reserved the device memory up
 * front (a further cudaMalloc would fail or fragment its pool), or a
 * latency-critical loop that cannot absorb the device-wide synchronisation of
 * cudaMalloc/cudaFree.  Same arguments and results as wpccc_matrix_elements
 * (S and H are written by the same kernels; the caller still owns them).
 * Scratch memory: a fixed array of WPCCC_NOALLOC_SCRATCH_BYTES (64 MiB) inside
 * the library, which every GPU that loads the library holds until the process
 * exits.  Nothing in it needs clearing (every byte a call reads it first writes),
 * and it keeps the last call's contents.  All calls on a device share it:
 * calls whose GPU work overlaps (other streams, other threads, other bases) race
 * and corrupt each other's results; serialise them.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process, so a cudaDeviceReset (or any
 * other end of the device's primary context) invalidates the library for that
 * device.  Positions are processed in groups that fit the array (at most 65535 per
 * group), and the call waits for each group with cudaStreamSynchronize(stream):
 * the call blocks, and it must not be issued while `stream` (or, for the legacy
 * default stream, any stream) is being captured into a CUDA graph.  Errors: EINVAL
 * (as wpccc_matrix_elements, or a basis whose single position needs more scratch
 * than the array holds; the message states both sizes), ECUDA.  The basis itself
 * must have been created beforehand.
 */
#define WPCCC_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
WPCCC_API wpccc_status wpccc_matrix_elements_noalloc(wpccc_basis basis, double b, double v, int nz,
                                                     const double* z, void* S, void* H, void* stream);

/*
 * Batched complex solve S X = H with partial pivoting (Sec. II: the paper calls
 * LAPACK/cuSOLVER/hipSOLVER ZGESV; this is a hand-written blocked LU).
 *   S     device [batch][N][N] complex128; overwritten by the factors L and U of
 *         P S = L U (unit lower L below the diagonal), as ZGETRF leaves them
 *   H     device [batch][N][N] complex128; overwritten by X (when info[k] == 0)
 *   ipiv  device [batch][N] int32; 1-based pivot rows as in LAPACK: row i was
 *         interchanged with row ipiv[i]
 *   info  device [batch] int32; 0 on success, k > 0 if U(k,k) is exactly zero (the
 *         factorisation is completed, H[k] holds no solution)
 *   precision_mode 0 = FP64 throughout (the only mode of this build)
 * The per-system outcome is only in `info`; the call itself returns OK once the
 * work is queued.  Errors: EINVAL (N < 1 or N > WPCCC_NMAX, batch < 0), EUNSUPPORTED
 * (precision_mode != 0), ECUDA.
 */
WPCCC_API wpccc_status wpccc_solve(int N, int batch, void* S, void* H, int* ipiv, int* info,
                         int precision_mode, void* stream);

/*
 * Propagates the amplitudes of every path through Algorithm 1: RK4 along the
 * path's z nodes with M = -(i/v) S^{-1} H evaluated at z, at the step midpoint
 * and at the next node (Eq. 2-4; Eq. 5, M = -(i/v) D_T, in one-centre mode).
 *   c  device [n_paths][N] complex128: in, the amplitudes at each path's first
 *      node (Algorithm 1 starts from c = (1, 0, ..., 0)); out, the amplitudes at
 *      its last node.
 *   precision_mode
 *     0  FP64 throughout;
 *     1  mixed: the Eq. 9 contraction and the LU factors of S on the FP32 pipe,
 *        each RK4 stage's S^{-1} solved by FP64 iterative refinement (residuals
 *        against the FP64 S), RK4 amplitudes in FP64;
 *     2  mixed with FP64 elements: as 1 but the contraction stays in FP64 (for
 *        ill-conditioned S, where FP32 element errors get amplified by cond(S));
 *     3  as 1 with the Eq. 9 contraction on the 5th-generation tensor cores: tcgen05.mma
 *        (kind::f16) on four bf16 fixed-point slices of both operands per 128-node window
 *        (ten slice products into four exact FP32 accumulators, about 2^-28 of each window's
 *        largest term), drained per window into double-float sums; table tiles staged by TMA;
 *     4  the FP64 form (solve and RK4 as mode 0) with the Eq. 9 contraction emulated to FP64
 *        accuracy on the tensor cores: seven bf16 slices of both operands in fixed point per
 *        128-node window (error-free splitting, Ozaki et al.), 28 slice products into five FP32
 *        accumulators of which four are exact, drained into double-float sums; element errors
 *        about 2^-47 of the largest quadrature term;
 *     5  as 2 (FP32 factors and FP64 refinement) with the elements of mode 4;
 *     modes 3-5 need no model potential and a node count that is a multiple of 128 (fixed-point
 *     scales per 128-node window); in one-centre mode all modes
 *     are the FP64 form (no contraction, no solve).
 *   batch_mode 0 = all paths batched together in chunks of RK4 steps (the only
 *   batch mode of this build).
 * Blocks until the work is finished: the library allocates its scratch memory
 * itself (kept with the basis for reuse) and checks the pivots and the
 * amplitudes at the end.
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM, ESINGULAR (some S had a zero pivot),
 * ENONFINITE (amplitudes became non-finite), ENOCONV (a refined mode's refinement did not converge, see
 * wpccc_basis_set_refine_tolerance), ETIMEOUT (a bounded wait of a kernel gave up), ECUDA.
 */
WPCCC_API wpccc_status wpccc_propagate(wpccc_basis basis, const wpccc_paths* paths, int precision_mode,
                             int batch_mode, void* c, void* stream);

/*
 * Batches: several sets of paths, each with its own basis (e.g. the same collision at several
 * speeds, with bases of different size and paths with different step counts), propagated together
 * by one CUDA graph launch.  The batch owns a plan per set (the positions of every chunk of RK4
 * steps, as wpccc_propagate uses them) and the device memory for all of them; creating it captures
 * every set's kernel sequence -- element kernels, solves and RK4 sweeps, the sets running
 * concurrently on their own streams -- into one graph.
 *   bases  host [n_sets] bases, all on one device; paths host [n_sets] path sets;
 *   c      host [n_sets] device pointers, set k's amplitudes [n_paths_k][N_k] complex128; the
 *          graph reads and writes them in place at every launch, so they must stay valid for
 *          the batch's lifetime;
 *   autotune  non-zero: for each set, time the default chunk schedule and chunks of half and
 *          twice as many RK4 steps on the set's first steps (on copies of c) and keep the fastest.
 * wpccc_batch_launch queues the graph on `stream` (asynchronous; one launch advances every set
 * through all its steps).  wpccc_batch_status waits on `stream` and reports ESINGULAR or
 * ENONFINITE from the last launch.  wpccc_batch_info gives each set's RK4 steps per chunk and the
 * autotuner's ms per step (0 when not tuned).  Errors: EINVAL, ENOMEM, ECUDA, as wpccc_propagate.
 */
typedef struct wpccc_batch_s* wpccc_batch;
WPCCC_API wpccc_status wpccc_batch_create(int n_sets, const wpccc_basis* bases, const wpccc_paths* paths,
                                          int precision_mode, void* const* c, int autotune, wpccc_batch* out);
WPCCC_API wpccc_status wpccc_batch_launch(wpccc_batch batch, void* stream);
WPCCC_API wpccc_status wpccc_batch_status(wpccc_batch batch, void* stream);
WPCCC_API wpccc_status wpccc_batch_info(wpccc_batch batch, int* chunk_steps, double* tuned_ms_per_step);
WPCCC_API wpccc_status wpccc_batch_destroy(wpccc_batch batch);

/*
 * Transition probabilities at the end of the paths (Sec. II: the solution at
 * z_max gives the observables): P[p][i] = |c[p][i]|^2.
 *   c  device [n_paths][N] complex128;  P  device [n_paths][N] double.
 * Errors: EINVAL, ECUDA.
 */
WPCCC_API wpccc_status wpccc_probabilities(int n_paths, int N, const void* c, double* P, void* stream);

/*
 * Observables at the end of the paths (Sec. II: the amplitudes at z_max give the transition
 * probabilities; capture sums the projectile's bound states, excitation a level's states):
 *   P[p][o] = sum_i g[o][i] |c[p][i]|^2.
 *   g  device [n_obs][N] real weights;  c  device [n_paths][N] complex128;  P  device [n_paths][n_obs].
 * Errors: EINVAL (n_paths < 0, N < 1, n_obs outside 1..65535, null pointers), ECUDA.
 */
WPCCC_API wpccc_status wpccc_observables(int n_paths, int N, int n_obs, const double* g, const void* c, double* P,
                                         void* stream);

/*
 * Cross sections sigma_o = 2 pi int_0^inf b P_o(b) db (Sec. II: the probabilities of all impact parameters
 * give the cross sections) by the trapezoid rule on the nodes 0, b[0], ..., b[n_b - 1] (b P(b) = 0 at b = 0):
 * sigma_o = sum_j 2 pi b_j w_j P[j][o], w_j = (b_{j+1} - b_{j-1}) / 2 with b_{-1} = 0 and, for the last node,
 * (b_{n-1} - b_{n-2}) / 2.
 *   b      host [n_b] impact parameters, finite, > 0, strictly increasing (1 <= n_b <= 2048)
 *   P      device [n_b][n_obs] observables of those paths;  sigma  device [n_obs]
 * Errors: EINVAL (sizes, unsorted or non-positive b, null pointers), ECUDA.
 */
WPCCC_API wpccc_status wpccc_cross_sections(int n_b, const double* b, int n_obs, const double* P, double* sigma,
                                            void* stream);

/*
 * Norms of the amplitudes at one position per path: out[p][0] = c_p^+ S(z_p) c_p and out[p][1] = c_p^+ c_p,
 * with S of Eq. 1 assembled at (b[p], v[p], z[p]) by the FP64 element kernels.  In the two-centre basis the
 * states are not orthogonal, so the probability the amplitudes carry is c^+ S c; with the lower-left block
 * of H taken as Q^+ (Eq. 1 as printed) the equations give d(c^+ S c)/dz = c^+ (dS/dz) c, so it is not an
 * invariant of the two-centre propagation (in one-centre mode S = I and both norms are c^+ c).
 *   b, v, z  host [n_paths];  c  device [n_paths][N] complex128;  out  device [n_paths][2] double
 * Blocks until done; allocates S and H for the positions (freed before it returns) and uses the basis
 * workspace.  Errors: EINVAL, ENOMEM, ECUDA.
 */
WPCCC_API wpccc_status wpccc_overlap_norms(wpccc_basis basis, int n_paths, const double* b, const double* v,
                                           const double* z, const void* c, double* out, void* stream);

/*
 * The basis' states in state order (every target state, then every projectile state): qn[i] = (centre:
 * 0 target, 1 projectile; radial function index on that centre; l; m) and eps[i] its energy (host arrays
 * [N][4] and [N]; either may be NULL).  Errors: EINVAL (null basis), ECUDA.
 */
WPCCC_API wpccc_status wpccc_basis_states(wpccc_basis basis, int* qn, double* eps);

/*
 * How wpccc_propagate applies S^{-1} (two-centre mode).  Both give M(z) c up to rounding.
 *   WPCCC_SOLVE_STAGE  (default) LU-factorise S(z) once per position; at every RK4
 *                      stage form H(z) y and solve S(z) k = H(z) y with the factors
 *                      ((8/3) N^3 flops per position plus 16 N^2 per stage).
 *   WPCCC_SOLVE_SCHUR  S = [[I, K], [K^+, I]] is Hermitian positive definite (a Gram matrix):
 *                      Cholesky-factorise its Schur complement I - K^+ K once per position
 *                      (4 N_P^2 N_T + (4/3) N_P^3 flops) and per stage solve
 *                      k_P = (I - K^+ K)^{-1} (t_P - K^+ t_T), k_T = t_T - K k_P (no pivoting;
 *                      a non-positive pivot is reported as ESINGULAR);
 *   WPCCC_SOLVE_MATRIX the paper's form: X = S^{-1} H with N right-hand sides per
 *                      position (ZGESV, (8/3 + 8) N^3 flops), then M c = -(i/v) X c.
 */
#define WPCCC_SOLVE_STAGE 0
#define WPCCC_SOLVE_MATRIX 1
#define WPCCC_SOLVE_SCHUR 2
WPCCC_API wpccc_status wpccc_basis_set_solve_mode(wpccc_basis basis, int mode);

/*
 * How the refined precision modes with WPCCC_SOLVE_SCHUR form their FP32 preconditioner's trailing matrix
 * I - K^+ K (the rank-N_T update that eliminates the identity block of S, the bulk of the factorisation):
 *   WPCCC_SCHUR_UPDATE_TENSOR      on the tcgen05 tensor cores as a real GEMM over the target index, both
 *                                  operands in four fixed-point bf16 slices per 128-wide window with exact
 *                                  FP32 level accumulators (about 2^-28 of each window's largest term), then
 *                                  the Cholesky factor on the CUDA cores;
 *   WPCCC_SCHUR_UPDATE_CUDA_CORES  update and Cholesky factor in FP32 on the CUDA cores, one block per
 *                                  position;
 *   WPCCC_SCHUR_UPDATE_AUTO        (default) tensor cores when N_P >= 256, else CUDA cores (below that the
 *                                  three launches of the tensor-core route cost more than they save).
 * Both are preconditioners of the same FP64 refinement; the tensor-core one is the more accurate (its
 * update carries no FP32 rounding), so the refinement converges faster.  Errors: EINVAL (null basis,
 * unknown mode).  The paper has no counterpart.
 */
#define WPCCC_SCHUR_UPDATE_AUTO 0
#define WPCCC_SCHUR_UPDATE_TENSOR 1
#define WPCCC_SCHUR_UPDATE_CUDA_CORES 2
WPCCC_API wpccc_status wpccc_basis_set_schur_update(wpccc_basis basis, int mode);

/*
 * Sweeps of FP64 iterative refinement per RK4 stage in the refined precision modes (1, 2, 3, 5):
 * x_0 from the FP32 factors, then x_{n+1} = x_n + S_32^{-1} (H y - S x_n) with the residual in FP64.
 * Each sweep shrinks the solve error by about cond(S) 2^-24; the default of 2 leaves it near
 * FP32-squared level, 3 to 4 reach FP64 rounding for well-conditioned S.  (The paper solves in
 * FP64 only; no counterpart.)  Errors: EINVAL (null basis, iters outside 1..WPCCC_MAX_REFINE).
 */
#define WPCCC_MAX_REFINE 8
WPCCC_API wpccc_status wpccc_basis_set_refine_iters(wpccc_basis basis, int iters);

/*
 * Convergence check of the refined precision modes (1, 2, 3, 5; the paper solves in FP64 only, no
 * counterpart): at every RK4 stage the last refinement sweep's correction dx is compared with the solution,
 * and wpccc_propagate returns WPCCC_ENOCONV if max|dx| > tol max|x| on any stage of any path (the sweeps
 * contract the error by a factor rho per sweep, so the error left after the last one is about rho max|dx|:
 * tol = 1e-3 bounds it near 1e-6 relative whenever rho < 1e-3, while a refinement that stalls or diverges,
 * rho >= 1, leaves max|dx| ~ max|x|).  Needs at least two sweeps (wpccc_basis_set_refine_iters).  tol <= 0
 * switches the check off.  Default 1e-3.  Errors: EINVAL (null basis, non-finite tol).
 */
WPCCC_API wpccc_status wpccc_basis_set_refine_tolerance(wpccc_basis basis, double tol);

/*
 * Iteration limit of every mbarrier wait in device code: the tensor-core kernels' waits (precision modes 3-5;
 * the contraction's TMA thread counts polls in which neither of its buffers came free) and the RK4 sweep's
 * waits for the bulk copies that stage H in shared memory (precision modes 1-3, N <= 512).  A tensor-core
 * CTA whose wait has polled `polls` times gives up, records the failure, lets the copies and tensor-core
 * operations it has in flight complete, frees its tensor memory and returns; an RK4 block records the
 * failure and goes on in step with its other threads, its copies landing before it returns.  The call then
 * reports WPCCC_ETIMEOUT and the device stays usable.  Default 2^20 polls (far longer than any wait of a
 * healthy launch).  A small limit makes the waits run out on purpose, to exercise that path.
 * Errors: EINVAL (null basis, polls < 1).
 */
#define WPCCC_DEFAULT_WAIT_POLLS (1L << 20)
WPCCC_API wpccc_status wpccc_basis_set_wait_limit(wpccc_basis basis, long polls);

/*
 * Where the RK4 sweep of Algorithm 1 keeps its vectors.
 *   WPCCC_RK4_SHARED  one thread block per path, c and the stage vectors in its shared memory, all the
 *                     chunk's steps in one launch (fastest; N up to about 2840 in the one-centre form,
 *                     fewer in the two-centre forms);
 *   WPCCC_RK4_GLOBAL  one-centre form only: one launch per RK4 stage for all paths of a chunk, the
 *                     matrix-vector product M(z) y spread over the GPU (a thread per row, the columns of
 *                     y staged in shared memory), the vectors in global memory; every chunk evaluates its
 *                     first node again instead of carrying the N x N matrix over (the paper's one-centre
 *                     runs at large l_max, N in the thousands);
 *   WPCCC_RK4_AUTO    (default) shared when it fits, else global.
 * Both give the same amplitudes up to rounding.  Errors: EINVAL (null basis, unknown layout).
 * EUNSUPPORTED from wpccc_propagate for WPCCC_RK4_GLOBAL with a two-centre basis.
 */
#define WPCCC_RK4_AUTO 0
#define WPCCC_RK4_SHARED 1
#define WPCCC_RK4_GLOBAL 2
WPCCC_API wpccc_status wpccc_basis_set_rk4_layout(wpccc_basis basis, int layout);

/*
 * Upper bound on the scratch memory wpccc_propagate may hold (default 8 GiB).
 * The number of RK4 steps batched per launch is chosen to fit it.
 */
WPCCC_API wpccc_status wpccc_basis_set_workspace_limit(wpccc_basis basis, size_t bytes);

/*
 * Kernel profiling of the work a basis queues (wpccc_matrix_elements,
 * wpccc_propagate and wpccc_propagate_adjoint): launches are always counted; when enabled, a pair of CUDA
 * events on the caller's stream brackets every launch and the device time is
 * accumulated per category.  Categories (WPCCC_PROF_N of them):
 *   0 node tables (Eq. 9 integrand factors), 1 molecular-frame contraction (Eq. 9),
 *   2 rotation (Eq. 8) and direct elements (Eq. 6), 3 linear solve (Eq. 4), 4 RK4,
 *   5 the adjoint kernels of wpccc_propagate_adjoint (reverse RK4 and element adjoint).
 * wpccc_profile_enable resets the counters.  wpccc_profile_read waits for the
 * recorded events and writes ms[WPCCC_PROF_N] (milliseconds, NULL to skip) and
 * launches[WPCCC_PROF_N] (NULL to skip).
 */
#define WPCCC_PROF_N 6
WPCCC_API wpccc_status wpccc_profile_enable(wpccc_basis basis, int on);
WPCCC_API wpccc_status wpccc_profile_read(wpccc_basis basis, double* ms, long long* launches);

/*
 * Differentiation form (no counterpart in the paper): derivatives of observables of the
 * propagated amplitudes with respect to n_par <= WPCCC_MAX_PARAMS parameters theta (e.g. the
 * projectile charge and the model-potential parameters).
 *
 * wpccc_basis_set_tangents gives the basis the derivatives of its inputs (host pointers, copied):
 *   dfT   [n_par][T.n_rad][Nr]  d f_a(r_i) / d theta_p of every target radial function
 *   depsT [n_par][T.n_rad]      d eps_a / d theta_p (every state of radial a shares it)
 *   dfP, depsP                  the same for the projectile centre
 *   dexplicit [n_par][4]        d(P.Z, mp_c, mp_a, mp_b) / d theta_p: how theta enters the
 *                               operator itself (projectile charge in D_T, target potential in Q
 *                               and D_P)
 * and builds, on the device, the derivative of the Eq. 7 table of each centre.  Synchronous.
 * Errors: EINVAL (one-centre basis, n_par out of range, null pointers), ENOMEM, ECUDA.
 */
#define WPCCC_MAX_PARAMS 4
WPCCC_API wpccc_status wpccc_basis_set_tangents(wpccc_basis basis, int n_par, const double* dfT,
                                                const double* depsT, const double* dfP, const double* depsP,
                                                const double* dexplicit);

/*
 * Observables P[p][o] = sum_i g[o][i] |c_i|^2 at the end of every path (Algorithm 1 in FP64,
 * stage-form solve) and their derivatives grad[p][o][k] = d P[p][o] / d theta_k, by the discrete
 * adjoint of the RK4 propagation: a forward sweep keeps the amplitudes every `checkpoint_every`
 * steps; the reverse sweep recomputes S, H and the amplitudes of one segment at a time and runs the
 * transposed RK4 stages backwards (S^-1 applied from the same LU factors), while the adjoint of the
 * element assembly contracts each stage's cotangent vectors with the derivatives of the element
 * integrals (the same Eq. 6-9 integrals with one radial table, the charge, the potential or the
 * energy phase differentiated).  The result is the exact derivative of the discrete propagation.
 *   n_obs  1..4 observables; g host [n_obs][N] real weights
 *   c      device [n_paths][N] complex128: in, amplitudes at the first node; out, at the last
 *   P      device [n_paths][n_obs] double, or NULL
 *   grad   device [n_paths][n_obs][n_par] double
 * Needs wpccc_basis_set_tangents first.  Two-centre bases only.  Blocks until done; allocates its
 * own checkpoint and segment buffers (freed before it returns) and uses the basis workspace.
 * Errors: EINVAL, EUNSUPPORTED (one-centre basis), ENOMEM, ESINGULAR, ENONFINITE, ECUDA.
 */
WPCCC_API wpccc_status wpccc_propagate_adjoint(wpccc_basis basis, const wpccc_paths* paths, int n_obs,
                                               const double* g, int checkpoint_every, void* c, double* P,
                                               double* grad, void* stream);

/* Text of the last error raised on the calling thread ("" if none). */
WPCCC_API const char* wpccc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WPCCC_H */
