/*
 * must.h -- C ABI of the GB300 LSMS tau_00 library.
 *
 * The library implements the hot path of the LSMS method as described in
 * arXiv 2308.16317 ("High Performance GPU Accelerated MuST Software"):
 *
 *   Eq. (4)   tau(E) = [t^{-1}(E) - g0(E)]^{-1}, with the KKR matrix
 *             M(E) = t^{-1}(E) - g0(E); g0 is the free-particle propagator
 *             between two *different* sites (Sec. 2.1).
 *   Sec. 2.1  rank of M is N (lmax+1)^2, or 2 N (lmax+1)^2 with spin canting.
 *   Sec. 2.2  LSMS builds M over the local interaction zone (LIZ) of each atom
 *             and needs only the first (central-site) block tau_00 of M^{-1}.
 *   Sec. 3.2  the paper inverts M by LU factorisation and solve; here M is
 *             assembled on the device and only tau_00 is formed.
 *   Sec. 5    building M on the GPU instead of the CPU is the paper's stated
 *             next step; it is what must_tau00_solve does.
 *
 * Conventions (Rydberg atomic units: lengths in bohr, energies in Ry):
 *   kappa = sqrt(E) on the principal branch (Im kappa > 0 for Im E > 0).
 *   L = l*l + l + m, m = -l..l; real spherical harmonics without the
 *   Condon-Shortley phase (Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x).
 *   g0^{ij}_{LL'} = -4 pi i kappa sum_L'' i^{l-l'+l''} C(L,L',L'')
 *                   h_l''(kappa |R_ij|) Y_L''(R_ij^),  R_ij = R_i - R_j.
 *   Complex numbers are interleaved (re, im) doubles.  tau_00 is returned
 *   column-major, kap x kap, kap = (lmax+1)^2 (2 (lmax+1)^2 when canted, with
 *   index (spin, L), spin up first).
 *
 * Memory: every pointer may be host or device memory unless stated; the
 * library detects which (cudaPointerGetAttributes) and stages host buffers
 * through the caller's workspace with stream-ordered copies.  The caller owns
 * all buffers, including the workspace; the library owns only the must_liz
 * handle and its device tables.  All GPU work is enqueued on the caller's
 * stream (a cudaStream_t passed as void*, NULL = legacy default stream).
 * Errors in arguments are returned synchronously; per-solve numerical
 * outcomes go to the optional per-solve status array.  No call throws.
 */
#ifndef MUST_H
#define MUST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MUST_OK = 0,
  MUST_EINVAL = 1,        /* bad argument (NULL, size, lmax, precision ...)      */
  MUST_ENOMEM = 2,        /* device allocation failed or workspace too small     */
  MUST_ECUDA = 3,         /* a CUDA runtime call failed (see must_last_error)    */
  MUST_ESINGULAR = 4,     /* per-solve: an exactly zero pivot was met            */
  MUST_ENOCONV = 5,       /* per-solve: refinement did not reach the tolerance   */
  MUST_ENONFINITE = 6,    /* per-solve: NaN/Inf in t^{-1} or in the result       */
  MUST_ETIMEOUT = 7,      /* a bounded device wait ran out                       */
  MUST_EUNSUPPORTED = 8   /* valid request this build does not support           */
} must_status;

typedef enum {
  MUST_FP64 = 0,          /* complex128 throughout (the paper's precision, Sec. 4.1) */
  MUST_MIXED_BF16X3 = 1,  /* FP32 factors, trailing updates as split-BF16x3 on the
                             tensor cores, FP64 residual refinement               */
  MUST_MIXED_TF32X3 = 2   /* as above with 3xTF32 trailing updates                */
} must_precision;

typedef struct {
  int32_t precision;      /* must_precision                                          */
  double tol;             /* refinement stop: ||delta X||_F <= tol ||X||_F (mixed); the
                             refinement also stops when corrections stop shrinking   */
  int32_t max_iter;       /* refinement iteration cap (mixed); 0 => MUST_ENOCONV     */
  int32_t warm_start;     /* reserved for the learned seed; 0 = cold solve           */
  int32_t deterministic;  /* 1 = static schedule in batched launches                 */
  int32_t equilibrate;    /* 1 = symmetric |diag M|^{-1/2} scaling before low-prec LU */
  int32_t residual;       /* mixed paths: how R = E0 - M X is formed (all ~2^-47 of
                             the row scale or better):
                             0 = FP64 (DFMA);
                             1 = double-float (unevaluated FP32 pairs, FP32 pipes);
                             2 = split-integer (leading 23 bits of M and X as
                                 integers, exact 64-bit products, FP32 remainders);
                             3 = tensor cores: M and X split into six fixed-point
                                 BF16 digits, digit products on tcgen05 with FP32
                                 accumulation that is exact over 128-element K
                                 chunks, chunks combined in integers (Ozaki-style
                                 error-free split); the diagonal entry in FP64.  */
} must_solve_opts;

typedef struct must_liz must_liz;   /* opaque, immutable after build */

/* Fill *opts with the defaults (FP64, tol 1e-10, max_iter 10, equilibrate 1,
   FP64 residual). */
void must_default_opts(must_solve_opts* opts);

/*
 * Build a LIZ handle (Sec. 2.2).  pos_bohr: n_sites x 3 site positions, row 0
 * is the central atom; species: n_sites ints in [0, n_species) selecting the
 * t^{-1} row used at each site; lmax in [0, 4]; spin_dirs: n_sites x 3 unit
 * vectors for the spin-canted matrix (rank 2 N (lmax+1)^2), or NULL for the
 * collinear one.  All three arrays are read on the host during the call.
 * Computes the device tables (pair geometry, Y_L of every pair direction,
 * Gaunt coefficients) on `stream` and returns after they are complete.
 * Errors: MUST_EINVAL (NULL, n_sites < 1, lmax out of range, coincident
 * sites, non-unit spin direction), MUST_ENOMEM, MUST_ECUDA.
 */
must_status must_liz_build(const double* pos_bohr, const int32_t* species, int32_t n_sites, int32_t lmax,
                           const double* spin_dirs, void* stream, must_liz** out);
void must_liz_free(must_liz* liz);

/* Matrix order n and block width kap of a handle. */
int32_t must_liz_order(const must_liz* liz);
int32_t must_liz_kappa(const must_liz* liz);

/*
 * Device workspace (bytes) that must_tau00_solve needs to process n_items
 * (energy, spin) matrices at once with the given options (opts NULL =
 * defaults).  A smaller workspace is accepted: the solve then processes the
 * items in chunks that fit, down to one matrix.
 */
size_t must_workspace_bytes(const must_liz* liz, int32_t n_items, const must_solve_opts* opts);

/*
 * Square-well single-site t^{-1}_l(E) (a fixture for the synthetic workloads,
 * not part of Eq. 4 itself): well depth V[p] inside r < r_mt, zero outside,
 * log-derivative matching of j_l(q r), q = sqrt(E - V), to j_l - i kappa t_l h_l.
 * E: nE complex; V: n_pot reals; out tinv: [n_pot][nE][lmax+1] complex.
 * Computed by a device kernel on `stream`; host pointers are staged.
 */
must_status must_tinv_square_well(int32_t nE, const double* E, int32_t n_pot, const double* V, double r_mt,
                                  int32_t lmax, double* tinv, void* stream);

/*
 * tau_00 = [M^{-1}]_00 for every energy and spin of one LIZ (Eq. 4, Sec. 2.2).
 *   E       : nE complex energies.
 *   tinv    : t^{-1}_l per [nspin][n_species][nE][lmax+1] complex.  Collinear
 *             handles produce one matrix per (spin, energy); canted handles
 *             need nspin == 2 (up, down in each site's local frame) and
 *             produce one matrix of order 2n per energy.
 *   tau00   : [n_out][nE][kap][kap] complex, column-major blocks, n_out = nspin
 *             (collinear) or 1 (canted).
 *   status  : optional int32 per output block (MUST_OK, MUST_ESINGULAR,
 *             MUST_ENOCONV, MUST_ENONFINITE), same order as tau00, or NULL.
 *   workspace / ws_bytes : caller-owned device memory (see
 *             must_workspace_bytes); must be 256-byte aligned.
 * The matrix is ordered with the central site last, so that eliminating the
 * leading n - kap columns (LU with partial pivoting restricted to those rows)
 * leaves the kap x kap Schur complement S with tau_00 = S^{-1}.
 * Returns after enqueueing (device pointers) or after the final copy (host
 * output pointers).  Errors: MUST_EINVAL, MUST_ENOMEM, MUST_ECUDA,
 * MUST_EUNSUPPORTED.
 */
must_status must_tau00_solve(const must_liz* liz, int32_t nE, const double* E, const double* tinv,
                             int32_t n_species, int32_t nspin, const must_solve_opts* opts, void* workspace,
                             size_t ws_bytes, double* tau00, int32_t* status, void* stream);

/*
 * Many LIZs in one call (the paper distributes atoms over MPI ranks, Sec. 4.2;
 * here all (LIZ, energy, spin) items of uneven order share launches).
 * lizs: n_liz handles (same lmax and canting).  E, tinv as for
 * must_tau00_solve, shared by every LIZ.  tau00: [n_liz][n_out][nE][kap][kap].
 * status: [n_liz][n_out][nE] or NULL.
 */
must_status must_tau00_batch(int32_t n_liz, const must_liz* const* lizs, int32_t nE, const double* E,
                             const double* tinv, int32_t n_species, int32_t nspin, const must_solve_opts* opts,
                             void* workspace, size_t ws_bytes, double* tau00, int32_t* status, void* stream);
size_t must_batch_workspace_bytes(int32_t n_liz, const must_liz* const* lizs, int32_t n_items_per_liz,
                                  const must_solve_opts* opts);

/*
 * Batched plan (the batched launch captured in a CUDA graph):
 * the complete launch sequence of one must_tau00_batch call with these
 * arguments is captured once into a CUDA graph; must_plan_launch replays it
 * on `stream`, so repeated solves with new contents in the same E / tinv
 * buffers (an SCF loop, a benchmark) pay no per-kernel launch cost.  All
 * pointers must be device memory and stay valid while the plan exists.
 * Plans with their own workspace, inputs and outputs are independent: two or
 * more may run at the same time on different streams (independent solves in
 * flight; the results equal those of one plan at a time bit for bit), which
 * keeps the GPU busy while one solve waits on its chain of panels.  One plan
 * must not be replayed on two streams at once (its buffers are shared).
 * Errors: MUST_EINVAL (host pointers, as for must_tau00_batch), MUST_ECUDA
 * (capture or instantiation failed).
 */
typedef struct must_plan must_plan;
must_status must_plan_batch(int32_t n_liz, const must_liz* const* lizs, int32_t nE, const double* E,
                            const double* tinv, int32_t n_species, int32_t nspin, const must_solve_opts* opts,
                            void* workspace, size_t ws_bytes, double* tau00, int32_t* status, must_plan** out);
must_status must_plan_launch(const must_plan* plan, void* stream);
void must_plan_free(must_plan* plan);

/*
 * Energy-contour integration of the site charge (the step after the path:
 * the charge of Eq. 2 from the site Green's function of Eq. 3).  Collinear
 * LIZs only.
 *
 * must_contour_weights: host arrays.  E [n_e] complex (re, im pairs): the
 * Gauss-Legendre nodes in the angle of the upper semicircle from e_bot to e_f
 * (theta = pi/2 (1 - x_k), from e_bot to e_f); w [n_e] complex: the weights of
 * int_{e_bot}^{e_f} f(E) dE along it, w_k = -(pi/2) W_k i r e^{i theta_k}.
 *
 * must_site_charge: for each of n_out output blocks s (the spins of one LIZ,
 * tau00 laid out as must_tau00_solve returns it, [n_out][nE][kap][kap]
 * column-major complex, kap = (lmax+1)^2), with the centre site a square
 * well of depth V[s] and radius r_mt:
 *   g_k    = int_sphere G(r, r; E_k) d^3r = sum_L tau_LL(E_k) F_l(E_k)
 *            - sum_l (2l+1) I_l(E_k),
 *   F_l = int_0^a Z_l^2 r^2 dr, I_l = int_0^a Z_l J_l r^2 dr, Z_l regular
 *   (j_l/t_l - i kappa h_l outside), J_l irregular (j_l outside);
 *   n_of_E[s][k] = -(1/pi) Im g_k (may be NULL); N[s] = -(1/pi) Im sum_k w_k g_k.
 * The sign is that of the retarded G of this library (g0 = -e^{i kappa d} /
 * (4 pi d)).  Every array must be device memory (MUST_EINVAL otherwise);
 * asynchronous on `stream`.
 */
/*
 * must_site_density: the spherically averaged charge density inside the
 * centre sphere at n_r radii r[i] (0 < r[i] <= r_mt; other radii give NaN),
 * for each output block s as in must_site_charge:
 *   n_of_r[s][i] = -(1/pi) Im sum_k w_k (1/(4 pi)) [sum_L tau_LL(E_k) Z_l(r_i)^2
 *                                               - sum_l (2l+1) Z_l(r_i) J_l(r_i)],
 * the angular average of the site Green's function G(r, r; E) of Eq. 3
 * integrated along the contour as in Eq. 2, so that 4 pi int_0^a n r^2 dr is
 * must_site_charge's N.  Inside the well Z_l = c_l j_l(q r) and J_l =
 * alpha_l j_l(q r) + beta_l y_l(q r), q = sqrt(E - V), matched at r_mt as
 * above.  Every array (E, w, V, tau00, r, n_of_r) must be device memory
 * (MUST_EINVAL otherwise); asynchronous on `stream`.
 */
must_status must_contour_weights(int32_t n_e, double e_bot, double e_f, double* E, double* w);
must_status must_site_charge(int32_t lmax, int32_t nE, const double* E, const double* w, int32_t n_out,
                             const double* V, double r_mt, const double* tau00, double* n_of_E, double* N,
                             void* stream);
must_status must_site_density(int32_t lmax, int32_t nE, const double* E, const double* w, int32_t n_out,
                              const double* V, double r_mt, const double* tau00, int32_t n_r, const double* r,
                              double* n_of_r, void* stream);

/*
 * Tuning knobs (set by the project's autotuner, paper_2308_16317_gb300/autotune.py):
 *   knob 0: sites per padding quantum when must_tau00_batch groups LIZs of
 *           uneven size (1..64, default 4);
 *   knob 1: complex columns per tensor-core tile of the trailing update
 *           (128 or 256, default 128);
 *   knob 2: trailing-update kernel for 128-column tiles (BF16 splits): the
 *           streamed kernels give each CTA a run of 64-column tiles with the
 *           U block resident and move C as follows: 3 (default) TMA loads
 *           into shared memory, results stored from registers; 2 loads and
 *           stores from registers; 1 TMA loads and stores through shared
 *           memory; 0 selects the one-CTA-per-tile kernel.  All streamed
 *           kernels give identical results;
 *   knob 3: longest run of row tiles per CTA of the streamed kernels (1..64,
 *           default 32; runs are split evenly, and shorter when few column
 *           tiles would leave SMs idle);
 *   knob 4: panel look-ahead of the mixed path: 1 (default) factors panel
 *           k+1 on a high-priority side stream while the rest of step k's
 *           trailing update runs, 0 keeps every step on the caller's stream;
 *   knob 5: right-hand sides per CTA of the mixed path's correction solve
 *           (2, 4 or 8; 0, the default, takes the most that fit: 8 up to
 *           order 3200, 4 up to 6400, 2 up to 12800) when knob 6 is 0;
 *   knob 6: correction solve kernel: 1 (default) thread-block clusters of
 *           CTAs per item and group of right-hand sides, the rows of L and U
 *           spread over the cluster and each solved 32-row block shared
 *           through distributed shared memory; 0 one CTA per item and group;
 *   knob 7: preferred CTAs per cluster of that kernel (2, 4 or 8, default 2;
 *           a larger cluster is taken when the rows do not fit its shared
 *           memory);
 *   knob 8: right-hand sides per cluster of that kernel (4, 8 or 16; 0, the
 *           default, takes the most whose rows fit 72 KB of shared memory);
 *   knob 9: U12 = L11^-1 A12 of the mixed path: 1 (default) persistent CTAs
 *           (contiguous runs of 64-column tiles, the next tile copied while
 *           the current one is multiplied), 0 one CTA per tile;
 *   knob 10: where the mixed path packs the A operand (L21 as BF16 hi/lo
 *           pairs) of each panel step: 0 a pack kernel on the caller's
 *           stream, 1 a pack kernel on the look-ahead's side stream, 2 the
 *           panel kernel itself; all three write the same values
 *           (default 0, the fastest on the 135-site LIZ);
 *   knob 11: paired panel steps of the mixed path: while the trailing block
 *           left after two panels has at least this many rows, the two
 *           steps' trailing updates are applied in one K = 128 pass (half
 *           the C traffic; the second panel then runs with nothing to
 *           overlap it).  0 pairs nothing; default 1536.  BF16 splits with
 *           knob 2 = 3 only;
 *   knob 12: shape of the cluster correction from the third correction on
 *           (CTAs per cluster * 100 + right-hand sides per cluster: 204, 404,
 *           408, 416, 804, 808, 816, ...; 0: the shape of the first two).
 *           Default 408;
 *   knob 13: kernel of the paired (K = 128) pass: 3 (default) C tiles
 *           loaded by TMA, 2 C through registers with a deeper A ring; both
 *           give identical results.
 * Process-wide; set them between calls, not while solves are being enqueued.
 */
must_status must_tune_set(int32_t knob, int32_t value);
int32_t must_tune_get(int32_t knob);

/*
 * Allocation-free FP64 solve.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run (their
 * device memory is owned by another allocator, or allocation is forbidden
 * where they call from), so they cannot supply the workspace that
 * must_tau00_solve needs.  It computes the same result as must_tau00_solve
 * with MUST_FP64 and default options, using a scratch array compiled into
 * the library: must_static_scratch_bytes() bytes (160 MiB, enough for one
 * energy of both spins at n = 2160) of device memory that every GPU which
 * loads the library holds until the process exits.  It calls no allocator.
 *   E, tinv, tau00, status : as for must_tau00_solve, but all must be device
 *                            memory (host buffers are rejected, MUST_EINVAL).
 * A LIZ whose one-energy working set exceeds the scratch is rejected with
 * MUST_EINVAL and a message naming the sizes.  The first call on each device
 * looks up the scratch address (cudaGetSymbolAddress) with that device
 * current; make it before any stream capture.  Every call shares the one
 * scratch array, which keeps the previous call's contents; calls whose GPU
 * work overlaps (other streams or host threads) race on it and must be
 * serialised by the caller.
 */
must_status must_tau00_solve_static(const must_liz* liz, int32_t nE, const double* E, const double* tinv,
                                    int32_t n_species, int32_t nspin, double* tau00, int32_t* status, void* stream);
size_t must_static_scratch_bytes(void);

/*
 * Learned warm start (an extension; the paper has no learned part).
 * A small MLP, three linear layers with SiLU between them, BF16 weights with
 * FP32 accumulation and FP32 master weights / Adam moments, trained and
 * evaluated by the library's own kernels.  It predicts tau_00(E_k) from
 * tau_00 at the neighbouring contour energies E_{k-1}, E_{k+1}, the three
 * energies, the spin and the LIZ's species occupancy; the prediction can seed
 * the refinement of must_tau00_solve_seeded, whose plain solve is the
 * fallback and the reference its error is measured against.
 *   must_mlp_create   n_in inputs, hidden width, n_out outputs, largest batch,
 *                     seed of the initial weights (device allocation).
 *   must_mlp_forward  y[batch][n_out] = net(x[batch][n_in]) (device FP32).
 *   must_mlp_gradients / must_mlp_train_step: mean over the batch of the
 *                     squared error against target[batch][n_out]; gradients
 *                     in the parameter layout W1[H][I] b1 W2[H][H] b2 W3[O][H]
 *                     b3 (host or device), loss as one double (host/device).
 *   must_mlp_get/set_params, must_mlp_save/load: FP32 master weights (and
 *                     Adam state for save/load; set_params resets Adam).
 *   must_mlp_features: x for n samples from tau_prev / tau_next
 *                     ([n][kap][kap] complex, device), E3 ([n][3] complex:
 *                     E_{k-1}, E_k, E_{k+1}), spin ([n] float, +-1), occupancy
 *                     ([n][n_occ] float); also the per-sample scale and the
 *                     interpolation (tau_prev + tau_next)/2.  n_in must equal
 *                     4 kap^2 + n_occ + 8.
 *   must_mlp_apply    tau_pred = interp + scale * y; must_mlp_targets the
 *                     inverse map (training targets from solved tau).
 */
typedef struct must_mlp must_mlp;
must_status must_mlp_create(int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch, uint64_t seed,
                            must_mlp** out);
void must_mlp_free(must_mlp* net);
size_t must_mlp_param_count(const must_mlp* net);
must_status must_mlp_get_params(const must_mlp* net, float* params, void* stream);
must_status must_mlp_set_params(must_mlp* net, const float* params, void* stream);
must_status must_mlp_forward(const must_mlp* net, int32_t batch, const float* x, float* y, void* stream);
must_status must_mlp_gradients(must_mlp* net, int32_t batch, const float* x, const float* target, float* grads,
                               double* loss, void* stream);
must_status must_mlp_train_step(must_mlp* net, int32_t batch, const float* x, const float* target, float lr,
                                double* loss, void* stream);
must_status must_mlp_save(const must_mlp* net, const char* path);
must_status must_mlp_load(must_mlp* net, const char* path);
must_status must_mlp_features(int32_t n, int32_t kap, const double* tau_prev, const double* tau_next,
                              const double* E3, const float* spin, const float* occ, int32_t n_occ, int32_t n_in,
                              float* x, float* scale, double* interp, void* stream);
must_status must_mlp_apply(int32_t n, int32_t kap, const float* y, int32_t n_out, const float* scale,
                           const double* interp, double* tau_pred, void* stream);
must_status must_mlp_targets(int32_t n, int32_t kap, const double* tau, const float* scale, const double* interp,
                             float* y, int32_t n_out, void* stream);

/*
 * Seeded solve (learned warm start).  As must_tau00_solve on a mixed-precision
 * path, but items with seed_mask[block] != 0 start the refinement from a
 * block column built from the predicted tau_seed[block] (kap x kap,
 * column-major, same indexing as tau00): X_c = tau_seed and, for every other
 * row, the single-scattering term X_i = -M_ii^{-1} sum_q M_{i,c q} tau_seed.
 * The seed is accepted only if ||E0 - M X||_F <= 1e-3 ||E0||_F; otherwise (and
 * for unmasked items) the plain low-precision solve starts the refinement,
 * which then runs to the same tolerance either way, so the plain solve is the
 * fallback and what the seed is checked against.  seed_used (optional) receives 1 where
 * the seed was accepted.  tau_seed, seed_mask, seed_used and tau00 must be
 * device memory.  Errors: as must_tau00_solve; MUST_EINVAL for MUST_FP64.
 */
must_status must_tau00_solve_seeded(const must_liz* liz, int32_t nE, const double* E, const double* tinv,
                                    int32_t n_species, int32_t nspin, const must_solve_opts* opts, void* workspace,
                                    size_t ws_bytes, const double* tau_seed, const int32_t* seed_mask, double* tau00,
                                    int32_t* status, int32_t* seed_used, void* stream);

/*
 * Instrumentation (not part of the paper's method).  When enabled, CUDA
 * events are recorded on the launching stream around each phase of the path
 * (0 assemble, 1 panel, 2 row_swap, 3 trsm, 4 pack, 5 trailing_update,
 * 6 schur_inverse, 7 residual, 8 correction, 9 other).  must_profile_read
 * waits for the recorded events (it synchronises the device), writes per
 * phase the summed milliseconds, the kernel launches and the matrix items
 * those launches processed (the refinement phases count only items that were
 * not yet converged) into ms / launches / items [n_phases] (any may be
 * NULL), clears them and returns the number of phases.  must_launch_count
 * returns the number of kernels this library has launched in the process.
 */
/*
 * Arithmetic peak probe (instrumentation, not part of the paper's method):
 * one launch of `blocks` CTAs of 256 threads keeping every lane busy with
 * independent chains of one instruction kind for `iters` iterations: kind 0
 * DFMA (a 4 x 4 register block, 16 chains per thread), 1 DMMA (mma.sync
 * m8n8k4 f64, 8 accumulators per warp), 2 FFMA (8 chains per thread).  sink: device memory of
 * blocks x 256 doubles (read for the chains' start values, overwritten with
 * their results).  *flops (host) receives the flops the launch performs; the
 * caller times the launch on `stream` and divides.  Errors: MUST_EINVAL
 * (kind, sizes, NULL or host sink), MUST_ECUDA.
 */
must_status must_peak_probe(int32_t kind, int32_t blocks, int64_t iters, double* sink, double* flops, void* stream);

/*
 * Full KKR of a periodic crystal (Sec. 5: the paper's next target is the
 * same matrix inverse in the original KKR method, with the KKR matrix built on
 * the GPU).  With N_b sites b_s in a cell of the lattice {R}, the structure
 * constants of Eq. (4) summed over the lattice with Bloch phases,
 *   G^{st}_{LL'}(k) = sum_{R: rho != 0} e^{ik.R} g0_{LL'}(rho),  rho = b_s - b_t - R,
 * give M(k) = t^{-1} - G(k) of rank N_b (lmax+1)^2 (Sec. 2.1), and the
 * site-diagonal block of tau in Eq. (4) is the Brillouin-zone average
 *   tau^{ss}(E) = (1/n_k^3) sum_k [M(k)^{-1}]^{ss}
 * over the Gamma-centred mesh k = sum_i (m_i / n_k) b*_i (b*_i the reciprocal
 * vectors, a_i . b*_j = 2 pi delta_ij).  The lattice sums are evaluated by
 * Ewald's split into a reciprocal-space and a real-space sum, both cut where
 * their Gaussian factor falls below e^{-40}; that cut holds for Re E <= 1.5 Ry
 * (items above it get MUST_EUNSUPPORTED in their status).  Everything is FP64.
 *
 * must_kkr_build: lattice: 3 x 3 row-major, rows a_1, a_2, a_3 (bohr); basis:
 * n_basis x 3 site positions (bohr), distinct modulo the lattice; site_class:
 * n_basis ints or NULL -- sites of one class are promised equal t^-1 in every
 * call (must_kkr_tau checks it and flags an item that breaks it with
 * MUST_EINVAL in its status); NULL makes every site its own class; lmax in
 * [0, 4] with n_basis (lmax+1)^2 <= 64 (one M(k) is inverted in one CTA's
 * shared memory) and at most 32 distinct site displacements b_s - b_t; n_k in
 * [1, 64]; eta: Ewald splitting parameter (bohr^-2), 0 = 4 pi / Omega^(2/3)
 * (0.7 of that with one site per cell), which keeps the two sums about equally
 * costly; the result does not depend on it, but below ~0.4 of that value the
 * factor e^{E/eta} starts to cost digits.  flags: 0, or MUST_KKR_NO_SYMMETRY
 * and/or MUST_KKR_NO_TABLE (below).  Without MUST_KKR_NO_SYMMETRY the
 * crystal's point group is used: the signed permutations g of the Cartesian
 * axes that map the lattice onto itself and each site onto a site of its class
 * (48 for the fcc lattice with one site, or the L1_2 cell with the corner in a
 * class of its own).  The diagonal blocks obey [M(gk)^{-1}]^{ss} = D(g)
 * [M(k)^{-1}]^{tt} D(g)^T, g b_t = b_s, with D(g) the real-harmonic
 * representation of g, so one point of each orbit of the mesh is inverted,
 * weighted by the orbit's size, and the sum is symmetrised,
 * tau^s = (1/|G|) sum_g D(g) S^{t} D(g)^T.  With the flag, or when only the
 * identity qualifies, one point of each pair {k, -k} is evaluated.  Host arrays,
 * read during the call.  Builds the k mesh, the reciprocal and real-space
 * vector lists and the Gaunt table on the device (synchronises `stream`).
 * Errors: MUST_EINVAL, MUST_ENOMEM, MUST_ECUDA.
 *
 * must_kkr_tau: n_items (<= 65535) independent (energy, potential) items.  E: n_items
 * complex; tinv: [n_items][n_basis][lmax+1] complex t^{-1}_l of each site;
 * tau: [n_items][n_basis][kap][kap] complex, column-major blocks, kap =
 * (lmax+1)^2; status: optional int32 per item (MUST_OK, MUST_ESINGULAR for an
 * exactly zero pivot in some M(k), MUST_ENONFINITE, MUST_EUNSUPPORTED) or NULL.
 * Pointers may be host or device memory (host buffers are staged through the
 * workspace); workspace: caller-owned device memory of at least
 * must_kkr_workspace_bytes(kkr, n_items) bytes (MUST_ENOMEM otherwise).
 * Asynchronous on `stream` for device outputs; returns after the final copy
 * for host outputs.  Errors: MUST_EINVAL, MUST_ENOMEM, MUST_ECUDA.
 *
 * must_kkr_info: info[9] = {M(k) order, k points evaluated, distinct
 * displacements, real-space points stored, (k, K) reciprocal terms, k groups,
 * mesh points n_k^3, real-space points of the zero displacement, point-group
 * operations used (0: k / -k pairing)}.  The
 * displacements x != 0 come in pairs (x, -x) and the real-space points of x = 0
 * in pairs (R, -R); one member of each is stored and summed for both.  In
 * the k / -k mode only one point of each pair {k, -k} of the mesh is
 * evaluated: M(-k) = M(k)^T (the reciprocity G_{LL'}(rho) = G_{L'L}(-rho)), so
 * its diagonal blocks enter the average transposed.  must_kkr_eta: the
 * splitting parameter in use.
 *
 * Reciprocal-term table: the factors of each reciprocal term that do not
 * depend on the energy (e^{-q^2/eta} YS_L(q), the phases cos(q.x) and sin(q.x)
 * of the displacements, q^2) are computed once by must_kkr_build and kept on
 * the device, 8 (2 lmax+1)^2 + 16 (number of displacement pairs) + 8 bytes per
 * (k, K) term (info[4] terms), when that is at most 512 MiB and the device
 * has room for it (otherwise the build goes on without it); every item of
 * must_kkr_tau then forms only 1/(q^2 - E) per term.  flags |=
 * MUST_KKR_NO_TABLE forms all factors per item instead (same results to
 * rounding).  must_kkr_table_bytes: the table's size, 0 when none is kept.
 *
 * must_kkr_geometry: the host half of must_kkr_build, with the same arguments
 * and checks but no device and no CUDA call: fills info[9] as must_kkr_info
 * would for the handle that build makes, and *eta_used (may be NULL) with the
 * splitting parameter.  Lets a host test the point group, the orbits of the
 * mesh and the vector lists without a GPU.  Errors: MUST_EINVAL.
 */
typedef struct must_kkr must_kkr;
#define MUST_KKR_NO_SYMMETRY 1   /* flags: evaluate one point of each {k, -k} pair only */
#define MUST_KKR_NO_TABLE 2      /* flags: form the reciprocal terms' harmonics per item, keep no table */
must_status must_kkr_build(const double* lattice, const double* basis, const int32_t* site_class, int32_t n_basis,
                           int32_t lmax, int32_t n_k, double eta, int32_t flags, void* stream, must_kkr** out);
void must_kkr_free(must_kkr* kkr);
size_t must_kkr_workspace_bytes(const must_kkr* kkr, int32_t n_items);
must_status must_kkr_tau(const must_kkr* kkr, int32_t n_items, const double* E, const double* tinv,
                         void* workspace, size_t ws_bytes, double* tau, int32_t* status, void* stream);
must_status must_kkr_info(const must_kkr* kkr, int32_t* info);
double must_kkr_eta(const must_kkr* kkr);
size_t must_kkr_table_bytes(const must_kkr* kkr);
must_status must_kkr_geometry(const double* lattice, const double* basis, const int32_t* site_class,
                              int32_t n_basis, int32_t lmax, int32_t n_k, double eta, int32_t flags,
                              int32_t* info, double* eta_used);

void must_profile_enable(int on);
int must_profile_read(double* ms, long long* launches, long long* items, int n_phases);
long long must_launch_count(void);
const char* must_phase_name(int phase);

const char* must_status_string(must_status s);
/* Message for the last non-OK status returned on the calling thread. */
const char* must_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MUST_H */
