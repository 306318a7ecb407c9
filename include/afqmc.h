/*
 * afqmc.h -- C ABI of the GB300 walker step of large-time-step phaseless AFQMC
 * (Sukurma, Schlipf, Humer, Taheridehkordi, Kresse: "Towards Large-Scale AFQMC
 * Calculations: Large Time Step Auxiliary-Field Quantum Monte Carlo").
 *
 * The library propagates a population of walkers.  A walker is a pair of
 * complex Slater determinants (alpha: N x na, beta: N x nb), a real weight W,
 * the complex log-overlap log <Psi_T|Psi> and a status word (Sec. II.A,
 * Eq. wavefun_rep).  One call of afqmc_step performs, for every walker:
 *   force bias with capping         (Eq. force_shift; Sec. V.C)
 *   field assembly                  (Eq. heffTOT)
 *   Split-2 propagation             (Sec. III.B) with the Taylor (Eq. taylor)
 *                                   or Krylov (Eqs. krylovsub-krylov) action
 *                                   of the one-body exponential; also the
 *                                   block-Krylov (Eq. bkrylov) and Chebyshev
 *                                   (Sec. IV.B) actions, and the Split-1,
 *                                   Taylor and Crank-Nicolson propagators
 *                                   (Sec. III.A, III.C, III.D)
 *   overlap ratio, hybrid energy    (Eqs. hyben, theta)
 *   phaseless weight with capping   (Eq. phaseless; Sec. V.B)
 *   optional re-orthonormalisation  (modified Gram-Schmidt per spin; the
 *                                   QR of Sec. IV.D, Psi = B_1 R, applied
 *                                   to the walkers)
 *   optional local energy, capping  (Eq. eloc, Eq. enwin) and the mixed
 *   and mixed estimator              estimator E_k (Sec. II.A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sizes: N orbitals, na/nb electrons per spin (nc = na + nb columns),
 *    G Cholesky vectors, Nw walkers.  1 <= N <= 512, 0 <= na, nb <= 80,
 *    1 <= na + nb <= N, 1 <= G; otherwise AFQMC_EINVAL.
 *  - Host matrices are row-major double.  h1[N*N] is the one-body matrix h_pq,
 *    L[G*N*N] the Cholesky vectors L_g,pq with <pq|rs> = sum_g L_g,pr L_g,qs
 *    (Sec. II.A), trial[nc*N] the trial orbitals stored orbital by orbital:
 *    trial[j*N + p] is coefficient p of orbital j; orbitals [0, na) are
 *    alpha, [na, nc) beta.  Host inputs are copied; the caller keeps
 *    ownership and may free them after the call returns.
 *  - Walker and field buffers are caller-owned DEVICE memory (for example
 *    PyTorch tensors); the library never frees them and uses them
 *    asynchronously on the context's stream.  The caller keeps them alive and
 *    unmodified until that stream has been synchronised.
 *  - psi[w][j][p] (w < Nw, j < nc, p < N) is interleaved complex: double2 for
 *    an AFQMC_FP64 context, float2 for an AFQMC_MIXED context; 16-byte
 *    (double) or 8-byte (float) alignment.
 *  - Every call returns a status; nothing throws, aborts or traps.  Numerical
 *    failure of a single walker (singular overlap, non-finite weight) sets its
 *    status bits and its weight to 0 instead of failing the call.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_ctx afqmc_ctx;  /* opaque; owned by the library */

typedef enum {
  AFQMC_OK = 0,
  AFQMC_EINVAL = 1,   /* null pointer, size out of range, unsupported value   */
  AFQMC_EDOM = 2,     /* non-finite host input (h1, L, trial, tau, e_const)    */
  AFQMC_ENOMEM = 3,   /* a device or host allocation failed                     */
  AFQMC_ECUDA = 4,    /* a CUDA runtime call failed; afqmc_last_cuda_error()    */
  AFQMC_ENOTSUP = 5,  /* propagator / exponential / precision not implemented   */
  AFQMC_ESTATE = 6    /* call out of order (e.g. a step before afqmc_set_tau)   */
} afqmc_status;

/* Propagators (Sec. III): Split-2, the paper's recommended one, Split-1, the
 * Taylor propagator and Crank-Nicolson. */
enum { AFQMC_SPLIT2 = 0, AFQMC_SPLIT1 = 1, AFQMC_TAYLORPROP = 2, AFQMC_CN = 3 };

/* Action of the one-body exponential (Sec. IV). */
enum {
  AFQMC_EXPM_TAYLOR = 0,
  AFQMC_EXPM_KRYLOV = 1,
  AFQMC_EXPM_BLOCK_KRYLOV = 2,
  AFQMC_EXPM_CHEBYSHEV = 3,
  AFQMC_EXPM_LANCZOS = 4
};

/* Arithmetic of a context.
 * AFQMC_FP64:  complex128 walkers, every step in FP64.
 * AFQMC_MIXED: complex64 walkers.  On the tensor cores in split BF16 (three
 *              bf16 products per FP32 operand pair, FP32 accumulation): the
 *              field assembly A = i sqrt(tau) sum_g c_g L_g, the products A*V
 *              of the Taylor and Krylov actions, the Split-2 half steps
 *              (Psi + (B - I) Psi, the identity part added in FP32) and the
 *              Coulomb + exchange contraction of E_L (whose Coulomb traces
 *              also give the force bias of the next step when reuse_bias is
 *              set).  In FP32: the overlap products trial^T Psi, O^{-1} from
 *              the rounded LU factors and Theta = Psi O^{-1}, the force-bias
 *              contraction when it is recomputed, the Arnoldi and Lanczos
 *              inner products, norms and square roots, the combinations of
 *              the Chebyshev recurrence, the shift A_w - tau h'' of the Taylor
 *              and Crank-Nicolson propagators, the one-body trace
 *              tr(h_half Theta) (error-free products and compensated
 *              TwoSum sums in FP32, per-thread partials added in FP64) and
 *              the Gram-Schmidt projections of the re-orthonormalisation (the
 *              walkers are stored in FP32; every result that depends on them
 *              is invariant under Psi -> Psi M, so the orthonormality of Q
 *              affects no energy or weight).  In FP64: the LU of the overlap
 *              matrices and their log-determinants, the small exponential
 *              e^{A_k} e_1 of the Krylov action, the Crank-Nicolson
 *              elimination, the hybrid energy, the
 *              phaseless weights, population control, and every sum over
 *              Cholesky vectors or walkers of the energies. */
enum { AFQMC_FP64 = 0, AFQMC_MIXED = 1 };

/* Per-walker status bits, OR-ed into status[w] (never cleared by the library). */
#define AFQMC_W_FCAP      0x1u  /* at least one force-bias component removed      */
#define AFQMC_W_REWEIGHT  0x2u  /* reweighting factor >= 10 set to 0 (Sec. V.B)  */
#define AFQMC_W_PHASE     0x4u  /* cos(dtheta) <= 0: killed by the phaseless cut */
#define AFQMC_W_NONFINITE 0x8u  /* non-finite ratio/energy/weight: weight set 0  */
#define AFQMC_W_SINGULAR  0x10u /* zero pivot in the overlap matrix; the weight
                                   update of the step gives such a walker W = 0 */

/* Walker population: caller-owned device buffers.
 *   psi     [Nw][nc][N] complex (see above)
 *   weight  [Nw] double, W >= 0; walkers with W == 0 are left untouched
 *   logovl  [Nw][2] double, (Re, Im) of sum_sigma log det(trial_s^T psi_s);
 *           the imaginary part is defined modulo 2*pi
 *   status  [Nw] uint32, AFQMC_W_* bits */
typedef struct {
  int n_walkers;
  void* psi;
  double* weight;
  double* logovl;
  uint32_t* status;
} afqmc_walkers;

/* Parameters of one step.
 *   tau         time step (> 0)
 *   e0          best estimate of the ground-state energy E_0 (Eq. imag_prop)
 *   propagator  AFQMC_SPLIT2 (Sec. III.B: e^{-tau H1/2} e^{A} e^{-tau H1/2}) or
 *               AFQMC_SPLIT1 (Sec. III.A: e^{-tau H1} e^{A}, the exponential first,
 *               then the one-body step applied as two half steps) or
 *               AFQMC_TAYLORPROP (Sec. III.C: the Taylor series of order `order` of
 *               e^{A - tau h''} applied to the walkers, no splitting; expm must be
 *               AFQMC_EXPM_TAYLOR, else AFQMC_ENOTSUP) or
 *               AFQMC_CN (Sec. III.D: (1 - X/2)^{-1} (1 + X/2) Psi with
 *               X = A - tau h'', by Gaussian elimination with partial pivoting
 *               per walker; expm and order are checked but not used; a
 *               singular 1 - X/2 leaves the walker non-finite, so the weight
 *               update kills it); other values: AFQMC_ENOTSUP
 *   expm        AFQMC_EXPM_TAYLOR (order = Taylor order 0 <= k <= 64),
 *               AFQMC_EXPM_KRYLOV (order = Krylov dimension 1 <= k <= 32, one
 *               Krylov space per orbital column, Eq. krylov),
 *               AFQMC_EXPM_LANCZOS (order = Krylov dimension 1 <= k <= 32; the
 *               same Krylov space per column, Eq. krylovsub, built by the
 *               complex-symmetric Lanczos recurrence, which the paper does
 *               not use: A is complex symmetric, so the bilinear form u^T v
 *               gives a basis V_k with V_k^T V_k = 1, the tridiagonal
 *               T_k = V_k^T A V_k and the action V_k e^{T_k} e_1 beta,
 *               beta = (psi^T psi)^{1/2}; three vectors read per step
 *               instead of the k of Arnoldi's Gram-Schmidt, no
 *               re-orthogonalisation, the recurrence stops when
 *               |beta_j| <= 1e-12 ||A||_F),
 *               AFQMC_EXPM_CHEBYSHEV (order = expansion order 0 <= k <= 64,
 *               Sec. IV.B: sum_n c_n T_n(A) Psi with c_0 = I_0(1),
 *               c_n = 2 I_n(1) and the recurrence of Eq. chebpoly, A not
 *               rescaled),
 *               AFQMC_EXPM_BLOCK_KRYLOV (order = number of blocks 1 <= k <= 16,
 *               Eq. bkrylov: per walker and spin, QR of the n orbitals, block
 *               Arnoldi with modified Gram-Schmidt, e^{A_k} E_n R of the
 *               (k n) x (k n) block Hessenberg; at most N / n blocks; the
 *               space is taken as invariant at the first new block whose QR
 *               has a diagonal entry <= 1e-12 ||A||_F).  ENOTSUP when the
 *               (k n)^2 + 3 (k n) n complex entries of the small exponential
 *               or the k n (n + N) of the combination do not fit one block's
 *               shared memory
 *   reortho     nonzero: re-orthonormalise every determinant (modified
 *               Gram-Schmidt) after the weight update and recompute logovl
 *   measure     nonzero: evaluate E_L at the new walkers (see
 *               afqmc_local_energy for the outputs)
 *   reuse_bias  nonzero: the mixed expectations <L_g> of the force bias (Eq.
 *               force_shift) are taken from the traces sum_s tr(Lh_gs Theta_s)
 *               of the last local-energy evaluation on this context when that
 *               evaluation was of the same walker buffers (psi pointer and
 *               count) and nothing changed the walkers since (a step,
 *               afqmc_walkers_init and afqmc_population_control invalidate
 *               it); Theta is invariant under re-orthonormalisation, so the
 *               quantity is the one the force bias would recompute.  The
 *               check runs on the device, so captured graphs honour it too.
 *               The caller must not modify the walkers between the two calls
 *               by other means.  0: always recompute. */
typedef struct {
  double tau;
  double e0;
  int propagator;
  int expm;
  int order;
  int reortho;
  int measure;
  int reuse_bias;
} afqmc_step_params;

/* Create a context for one Hamiltonian (Sec. II.A, Eq. mbham in Cholesky form)
 * and trial determinant.  Computes on the device the mean-field shift
 * L_bar_g = <Psi_T|L_g|Psi_T> (Eq. force_shift), the half-rotated vectors
 * trial^T L_g, trial^T h1, the propagation one-body matrix
 * h'' = h1 - 1/2 sum_g L_g L_g + sum_g L_bar_g L_g and its eigendecomposition
 * (host, FP64 Jacobi), used for e^{-tau h''/2} (Sec. III.B).
 *   out        receives the context
 *   precision  AFQMC_FP64 or AFQMC_MIXED
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 * Errors: EINVAL (sizes/pointers), EDOM (non-finite input), ENOMEM, ECUDA. */
afqmc_status afqmc_create(afqmc_ctx** out, int N, int n_alpha, int n_beta, int n_chol,
                          const double* h1, const double* L, const double* trial,
                          double e_const, int precision, void* stream);

/* Set the time step: uploads B = e^{-tau h''/2} (Sec. III.B, computed exactly
 * from the eigendecomposition).  afqmc_step calls it itself when its tau
 * differs from the current one; call it before capturing steps in a CUDA
 * graph.  Errors: EINVAL/EDOM (tau <= 0 or non-finite), ECUDA. */
afqmc_status afqmc_set_tau(afqmc_ctx* ctx, double tau);

/* Run subsequent work on another stream (cudaStream_t). */
afqmc_status afqmc_set_stream(afqmc_ctx* ctx, void* stream);

/* Psi_0 = Psi_T, W_0 = 1, logovl = log <Psi_T|Psi_T>, status = 0 (Sec. II.A). */
afqmc_status afqmc_walkers_init(afqmc_ctx* ctx, const afqmc_walkers* w);

/* One phaseless walker step of the whole population (see the file comment).
 *   fields   device [Nw][G] double, standard-normal auxiliary fields x_g^w
 *            (Eq. hstrafo); read only
 *   e_loc    device [Nw][2] double (Re, Im of E_L) or NULL; written when
 *            p->measure is nonzero (for walkers whose weight was already 0
 *            before the step the value is unspecified)
 *   e_mix    device [4] double or NULL; written when p->measure is nonzero:
 *            { sum_w W E_L_capped, sum_w W, E_k = ratio, live walkers }
 * The context keeps scratch space sized for the largest Nw seen; a larger Nw
 * reallocates it (do that before any graph capture).
 * Errors: EINVAL, ENOTSUP (propagator/expm/order), ECUDA, ENOMEM. */
afqmc_status afqmc_step(afqmc_ctx* ctx, const afqmc_walkers* w, const double* fields,
                        const afqmc_step_params* p, double* e_loc, double* e_mix);

/* Local energy E_L = <Psi_T|H|Psi>/<Psi_T|Psi> of every walker (Eq. eloc),
 * the capped value of Eq. enwin with DeltaE = 1/2 sqrt(N_e/tau) + sqrt(N_e tau)
 * around e0, and the mixed estimator E_k = sum W E_L_capped / sum W over
 * walkers with W > 0 (Sec. II.A).  Outputs as for afqmc_step.
 * Errors: EINVAL, ECUDA, ENOMEM. */
afqmc_status afqmc_local_energy(afqmc_ctx* ctx, const afqmc_walkers* w, double e0, double tau,
                                double* e_loc, double* e_mix);

/* Population control by comb resampling.  The paper does not describe one;
 * the comb is the reading taken: with cumulative weights
 * C_w = W_0 + ... + W_w summed in walker order in FP64, tooth j at
 * (u + j) C_{Nw-1} / Nw selects the first walker w with C_w > tooth (walkers
 * with W = 0 are never selected).  The population is replaced in place: slot j
 * receives a copy of its selected walker (psi, logovl, status) and every
 * weight becomes C_{Nw-1} / Nw, so the total weight is kept.
 *   u          caller-supplied uniform number in [0, 1)
 *   index_out  device [Nw] int32 or NULL: the source walker of every slot
 * If the total weight is not positive and finite the walkers are left
 * unchanged and index_out (when given) is filled with -1; the call itself
 * runs asynchronously on the context's stream.
 * Errors: EINVAL (u outside [0, 1), bad buffers), EDOM (u not finite), ECUDA. */
afqmc_status afqmc_population_control(afqmc_ctx* ctx, const afqmc_walkers* w, double u, int32_t* index_out);

/* Autotuner of the step's GEMM tile shapes.  Every walker-batched GEMM call
 * site of afqmc_step (force bias, field assembly, half step B*Psi, products
 * A*V of the exponential) has output-tile variants 0..3 (64x64, 128x32,
 * 32x128, 64x32) and variant 4, a per-walker kernel holding all orbital
 * columns of a walker (used where it applies, i.e. for A*V; elsewhere it
 * falls back to variant 0); this call times each variant at each site with CUDA events
 * (one warm-up, three timed launches, minimum kept) for n_walkers walkers on
 * the context's workspace and keeps the fastest.  Tile shape does not change
 * the summation order, so results are bit-identical for every choice.  (Mixed
 * contexts run their half steps on the tensor cores, or, where that plan is
 * unavailable and N <= 128, in a dedicated kernel that keeps B in shared
 * memory; the half-step site's choice then serves the adjoint.)
 * Synchronises the context's stream.
 *   table_out  host [4] int32 or NULL: the chosen variant per call site.
 * afqmc_tune_set / afqmc_tune_get write / read that table (e.g. from a cache
 * file).  Errors: EINVAL (bad table), ENOMEM, ECUDA. */
afqmc_status afqmc_autotune(afqmc_ctx* ctx, int n_walkers, int32_t* table_out);
afqmc_status afqmc_tune_set(afqmc_ctx* ctx, const int32_t* table);
afqmc_status afqmc_tune_get(const afqmc_ctx* ctx, int32_t* table);

/* A batch of independent systems (uneven N, electrons, G and walker counts)
 * stepped together.  Each afqmc_batch_step runs afqmc_step for every system
 * as one CUDA graph in which every system is a parallel branch between one
 * fork and one join, so small systems share the GPU.  The graph is captured
 * on the first call with a given set of arguments (walker buffers, field
 * pointers, step parameters, output pointers; up to four such sets are
 * cached) and replayed afterwards: to advance in time, write the next fields
 * into the same field buffers.  A capture first sets the time step and sizes
 * each context's workspace outside the capture.
 *   ctxs     [n_sys] contexts (they must outlive the batch)
 *   ws       [n_sys] walker sets; fields [n_sys] device pointers as for
 *            afqmc_step; p [n_sys] step parameters; e_loc, e_mix: NULL or
 *            [n_sys] device pointers (entries may be NULL)
 *   stream   cudaStream_t on which the graph is launched
 * Errors: as afqmc_step, plus ECUDA for a failed capture. */
typedef struct afqmc_batch afqmc_batch;
afqmc_status afqmc_batch_create(afqmc_batch** out, afqmc_ctx* const* ctxs, int n_sys);
afqmc_status afqmc_batch_step(afqmc_batch* batch, const afqmc_walkers* ws, const double* const* fields,
                              const afqmc_step_params* p, double* const* e_loc, double* const* e_mix,
                              void* stream);
void afqmc_batch_destroy(afqmc_batch* batch);

/* Adjoint of the mixed energy estimator at fixed walkers and weights.  The
 * paper has no gradients; this serves energy derivatives such as bond-length
 * scans.  With M_ws = Theta_ws trial_s^T the local energy of Eq. eloc is
 * E_const + sum_s tr(h1 M_ws) + 1/2 sum_g [(sum_s tr(L_g M_ws))^2
 * - sum_s tr(L_g M_ws L_g M_ws)], so for E_k = sum_w W Ebar_L / sum_w W
 * (Sec. II.A; dEbar/dRe E_L = 1 strictly inside the window of Eq. enwin,
 * 0 outside; walkers with W = 0 excluded):
 *   grad_h1  = dJ * Re sum_w c_w sum_s trial_s Theta_ws^T          [N][N]
 *   grad_L_g = dJ * Re sum_w c_w sum_s trial_s (t_wg I - T_wgs^T) Theta_ws^T
 * with c_w = W_w / sum W, T_wgs = trial_s^T L_g Theta_ws, t_wg = sum_s tr T_wgs.
 * Derivatives are with respect to every entry of h1 and L_g (a symmetric
 * direction dH gives sum_pq dH_pq grad_pq).  The trial is held fixed.
 *   grad_h1  device [N][N] double, grad_L device [G][N][N] double (written)
 * Both precisions: in a mixed context Theta and the per-walker terms are
 * complex64 (FP32 contractions over N) and the sums over walkers FP64.
 * AFQMC_ENOTSUP when na*na + na*N complex doubles exceed one block's shared
 * memory.  Synchronises the stream.
 * Errors: EINVAL, EDOM, ENOTSUP, ENOMEM, ECUDA. */
afqmc_status afqmc_energy_backward(afqmc_ctx* ctx, const afqmc_walkers* w, double e0, double tau, double dJ,
                                   double* grad_h1, double* grad_L);

/* Adjoint of a fixed-field walk: gradient of the mixed estimator after n steps,
 * J = E_n = sum_w W_n Ebar_L(Psi_n) / sum_w W_n (Sec. II.A), with respect to h1
 * and every L_g, through every step of the walk (Split-2 propagator, Sec. III.B,
 * with the Taylor exponential of Eq. taylor or the Krylov action of Eqs.
 * krylovsub-krylov, differentiated through its Arnoldi (or complex-symmetric
 * Lanczos) steps, norms and small exponential).  The paper has no gradients; the
 * readings taken are: the auxiliary fields are fixed inputs; every threshold
 * decision of the forward walk (force-bias removal |f_g| >= 1, reweighting cap,
 * cos(dtheta) <= 0, energy window) is held fixed, so a removed component or a
 * capped quantity carries no derivative, and d max(0, cos dtheta) =
 * -sin(dtheta) d(dtheta) where cos > 0; the re-orthonormalisation is a fixed
 * right multiplication Psi <- Psi R^{-1} (exact for the Taylor action: E_L,
 * the force bias, the overlap ratio and that action are invariant under
 * Psi -> Psi M; a column-wise Krylov or Lanczos action of dimension k < N is
 * not, so with re-orthonormalisation the gradient leaves out the part of dJ
 * that flows through R, a term of the order of the Krylov truncation);
 * the trial is held fixed; the dependence of e^{-tau h''/2} on h'' is taken
 * through the eigendecomposition (Daleckii-Krein divided differences).  The
 * mean-field shift L_bar_g = <Psi_T|L_g|Psi_T>, h'' and E_c' are functions of
 * h1 and L and are differentiated as such.
 * The walk is recomputed from checkpoints taken every ckpt_every steps.
 *   initial   walkers at step 0 (read only; logovl must equal
 *             log <Psi_T|Psi_0>, as afqmc_walkers_init leaves it)
 *   fields    device [n_steps][Nw][G] double, the fields of each step
 *   p         n_steps >= 1; expm = AFQMC_EXPM_TAYLOR (order = Taylor order
 *             1..32), AFQMC_EXPM_KRYLOV or AFQMC_EXPM_LANCZOS (order =
 *             Krylov dimension 1..32, taken as min(order, N); an invariant
 *             subspace found by a column ends its basis as in the step, the
 *             threshold held fixed; the Lanczos recurrence is holomorphic,
 *             so its square roots are differentiated on their principal
 *             branch), other values AFQMC_ENOTSUP; reortho_every r:
 *             re-orthonormalise after step k when (k+1) % r == 0 (0: never);
 *             ckpt_every >= 1; tau > 0; e0; dJ scales every output gradient
 *   J_out     device [4] double or NULL: {sum W Ebar_L, sum W, J, live
 *             walkers} after the walk (as e_mix of afqmc_step)
 *   grad_h1   device [N][N] double, grad_L device [G][N][N] double (written):
 *             dJ times the derivative along symmetric perturbations, returned
 *             symmetrised (for a symmetric direction dH the change of J is
 *             sum_pq dH_pq grad_pq)
 *   grad_psi0 device [Nw][na+nb][N] of the walkers' complex type, or NULL:
 *             G with dJ = Re sum G * dPsi_0 element by element (no
 *             conjugation), for a change of the initial walkers with logovl
 *             following Psi_0
 * Precision: an FP64 context runs everything in FP64.  A mixed context walks
 * its complex64 walkers with its own step (tensor-core field and Taylor
 * products) and runs the reverse pass on complex64 states and adjoints with
 * FP32 contractions; the overlap inverses, log-determinants, weights and the
 * per-walker coefficients are FP64, and the gradient sums over walkers and
 * steps are kept in FP64 (each step's complex64 contribution is added once).
 * The recomputed steps use the SIMT FP32 contractions, so they follow the
 * forward walk to FP32 rounding.
 * Memory: the call allocates and frees its own device workspace (about
 * (ckpt_every + n_steps/ckpt_every + 2 order + 12) Nw (na+nb) N complex
 * numbers of the walkers' type plus Nw N^2 of them, G N^2 complex doubles
 * and, in mixed contexts, G N^2 + G (na+nb) N complex floats; the Krylov
 * action adds Nw (na+nb) N more of the walkers' type and, for each of the
 * Nw (na+nb) columns, a copy of its k x k Hessenberg block in the walkers'
 * type plus k^2 + k + 2 complex doubles for the block's adjoint).
 * AFQMC_ENOTSUP when max(na, nb) > 64.  Synchronises the stream.
 * Errors: EINVAL, EDOM, ENOTSUP, ENOMEM, ECUDA. */
typedef struct {
  int n_steps;
  int order;
  int reortho_every;
  int ckpt_every;
  double tau;
  double e0;
  double dJ;
  int expm;
} afqmc_walk_adjoint_params;
afqmc_status afqmc_walk_backward(afqmc_ctx* ctx, const afqmc_walkers* initial, const double* fields,
                                 const afqmc_walk_adjoint_params* p, double* J_out, double* grad_h1,
                                 double* grad_L, void* grad_psi0);

/* Size of the device scratch array used by afqmc_local_energy_static. */
#define AFQMC_STATIC_SCRATCH_BYTES ((unsigned long long)32 << 20) /* 32 MiB */

/* afqmc_local_energy without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc when they need energies -- code running while a framework's
 * caching allocator owns the device memory, code held to a memory budget
 * fixed at start-up, or code that must not let an allocation synchronise
 * the device.  afqmc_local_energy may grow the context's workspace with
 * cudaMalloc; this variant instead uses one file-scope device array of
 * AFQMC_STATIC_SCRATCH_BYTES that the CUDA runtime reserves on every device
 * that loads the library and keeps until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine and runs the same kernels,
 * so its outputs equal those of afqmc_local_energy.
 *   e_loc, e_mix  caller-owned device outputs, as for afqmc_local_energy,
 *                 both required (non-NULL).
 * Scratch needed, each term rounded up to a multiple of 256 bytes:
 *   Nw*nc*N*c (c = 16 for FP64, 8 for mixed contexts) + Nw*32 + Nw*128
 *   + Nw*G*64 + Nw*8 bytes, plus 2 * (8*Nw*na*Kp) bytes (Kp = N rounded up to
 *   a multiple of 64) for mixed contexts whose exchange term runs on the
 *   tensor cores (every mixed context with 1 <= na == nb <= 64, whatever N);
 *   a call needing more than AFQMC_STATIC_SCRATCH_BYTES returns AFQMC_EINVAL
 *   and launches nothing.
 * The call must be made with the context's device current (the device that
 * was current at afqmc_create); from any other device it returns
 * AFQMC_EINVAL and launches nothing.
 * The first call on a device looks up the array's device address on the
 * current device (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls share the one array and it keeps the contents of
 * the last call; every value a call reads there is written by the same call
 * first, so nothing needs clearing.  Calls whose work overlaps on the GPU
 * (different streams, contexts or host threads without ordering) race on the
 * array and give wrong results.
 * Errors: EINVAL (null outputs, misaligned buffers, too large, not the
 * context's device), EDOM, ECUDA. */
afqmc_status afqmc_local_energy_static(afqmc_ctx* ctx, const afqmc_walkers* w, double e0, double tau,
                                       double* e_loc, double* e_mix);

/* Block until the context's stream is idle; returns ECUDA on a pending error.
 * Every wait of the tensor-core pipelines (TMA, MMA, TMEM hand-offs) gives up
 * after about 2 s; the kernel then raises the context's timeout flag, drains
 * what it issued, frees its TMEM and returns.  afqmc_sync reports a raised
 * flag as ECUDA (afqmc_last_cuda_error names the pipeline and the stage bits)
 * and clears it, so the next call starts clean. */
afqmc_status afqmc_sync(afqmc_ctx* ctx);

/* Check of the bounded waits above: one kernel waits for an mbarrier phase
 * that nothing completes, with the pipelines' wait helper bounded by
 * limit_cycles (1 .. 4e9 SM cycles, about 2 s at the top clock), then raises
 * bit 128 of the context's tensor-core timeout flag and returns; the next
 * afqmc_sync reports it.  The paper has no counterpart: this exists so that
 * the timeout path can be exercised without a GPU fault.  Nothing else is
 * launched or left in flight.
 * Errors: EINVAL (limit out of range), ENOTSUP (no tensor-core exchange in
 * this context, i.e. not a mixed context with 1 <= na == nb <= 64), ECUDA. */
afqmc_status afqmc_wait_probe(afqmc_ctx* ctx, long long limit_cycles);

/* Kernel classes of the per-class timer. */
enum {
  AFQMC_K_EXCHANGE = 0,   /* Coulomb + exchange contraction of E_L            */
  AFQMC_K_FIELD = 1,      /* field assembly A = i sqrt(tau) sum_g c_g L_g      */
  AFQMC_K_EXPM = 2,       /* products A*V of the Taylor / Krylov action        */
  AFQMC_K_FORCEBIAS = 3,  /* <L_g>_mixed contraction                           */
  AFQMC_K_HALFSTEP = 4,   /* B*Psi, B = e^{-tau h''/2}                         */
  AFQMC_K_OVERLAP = 5,    /* overlap, LU, log det, Theta                       */
  AFQMC_K_OTHER = 6,      /* everything else                                   */
  AFQMC_K_COUNT = 7
};

/* Per-class launch timing.  enable != 0 clears the accumulators and starts
 * recording a CUDA event before and after every launch on the context's
 * stream (at most 32768 launches; later ones are not recorded); enable == 0
 * stops.  afqmc_profile_read synchronises the stream, folds the recorded
 * event pairs into the accumulators and returns, per class, the summed
 * milliseconds ms[AFQMC_K_COUNT] and the number of launches n[AFQMC_K_COUNT].
 * afqmc_profile_mask does the same for the classes whose bit (1 << class) is
 * set in mask and records nothing around the other launches (mask 0 stops;
 * afqmc_profile(ctx, 1) is afqmc_profile_mask(ctx, (1 << AFQMC_K_COUNT) - 1)),
 * so that one kernel class can be timed inside a run without event pairs
 * around every other launch.
 * Errors: EINVAL (also: mask bits beyond AFQMC_K_COUNT), ENOMEM, ECUDA. */
afqmc_status afqmc_profile(afqmc_ctx* ctx, int enable);
afqmc_status afqmc_profile_mask(afqmc_ctx* ctx, uint32_t mask);
afqmc_status afqmc_profile_read(afqmc_ctx* ctx, double* ms, uint64_t* n);

/* Number of kernel launches the context has issued so far. */
uint64_t afqmc_launch_count(const afqmc_ctx* ctx);

/* Release the context and its device memory (NULL is ignored). */
void afqmc_destroy(afqmc_ctx* ctx);

const char* afqmc_strerror(afqmc_status s);

/* Host utility: eigendecomposition of a real symmetric n x n matrix a
 * (row-major, not modified) by cyclic Jacobi rotations in FP64; on return
 * evals[k] and column k of evecs (row-major n x n) form an eigenpair.  The
 * contexts use it for h'' when building e^{-tau h''/2} (Sec. III.B, "computed
 * exactly by diagonalisation").  Errors: EINVAL (n < 1, null), EDOM. */
afqmc_status afqmc_host_eigh(int n, const double* a, double* evals, double* evecs);

/* Text of the last CUDA error seen on the calling thread. */
const char* afqmc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
