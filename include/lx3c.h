/*
 * lx3c — 3-center Coulomb integrals (ab|C) and density-fitted Coulomb (DF-J)
 * quantities on one NVIDIA GB300 (sm_103a), all arithmetic in FP64.
 *
 * Method: Asadchev & Valeev, "Memory-Efficient Recursive Evaluation of
 * 3-Center Gaussian Integrals" (arXiv:2210.03192):
 *   Boys function -> [00|0]^(m) (Sec. 2.5.2) -> VRR1 (Eq. vrr1) ->
 *   early-contracted n-quantum CVRR2 (Sec. 2.5.4, Eqs. a0cv2/cVRR2) ->
 *   Cartesian-to-solid-harmonic ket transform -> HRR (Eq. hrr),
 *   and integral digestion into DF-J (Sec. 3): gamma_P = sum_ab (ab|P) D_ab,
 *   J_ab = sum_P (ab|P) c_P.
 *
 * Conventions (all calls):
 *   - Primitive Gaussians are NOT normalised (paper, Appendix A); contraction
 *     coefficients are used exactly as given.
 *   - Units: bohr.  Shell l <= LX3C_LMAX_ORB for orbital (bra) shells and
 *     l <= LX3C_LMAX_AUX for auxiliary (ket) shells; at most LX3C_KMAX
 *     primitives per shell.
 *   - Cartesian order inside a shell: x descending, then y descending
 *     (xx, xy, xz, yy, yz, zz).  Solid harmonics: real, Racah-normalised,
 *     ordered m = -l..l (p: y, z, x); S_{l,0}(0,0,1) = 1.
 *   - The ket shell is always solid harmonic.  The bra is solid harmonic when
 *     bra_pure != 0 (each bra shell projected like the ket), else Cartesian.
 *   - Integral block layout: out[pair][aux][A][B][C], C fastest, row-major,
 *     FP64, pairs and aux shells in the caller's list order.
 *   - Ownership: caller owns every data buffer it passes; the library owns
 *     lx3c_basis / lx3c_plan objects, freed with the matching destroy call.
 *   - Pointers marked "device" must be device (HBM) pointers of the current
 *     device; "host" pointers are read (or written) before the call returns.
 *   - Streams: `stream` is a cudaStream_t passed as void* (0 = legacy default
 *     stream).  Execute calls are asynchronous on that stream; *_create and
 *     *_plan calls may synchronise.
 *   - Errors: every call returns an lx3c_status; on failure nothing is
 *     launched (input is validated on the host first) unless the status is
 *     LX3C_ECUDA.  lx3c_last_error() returns a thread-local message.
 */
#ifndef LX3C_H
#define LX3C_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lx3c_status;
#define LX3C_OK 0
#define LX3C_EINVAL (-1)   /* malformed argument (null pointer, bad index, mixed class, ...) */
#define LX3C_ENOTSUP (-2)  /* outside supported limits (l, K, shared-memory budget) */
#define LX3C_ENOMEM (-3)   /* host or device allocation failed */
#define LX3C_ECUDA (-4)    /* a CUDA runtime call failed */
#define LX3C_EDEVICE (-5)  /* a kernel reported an error through its status word */

#define LX3C_LMAX_ORB 6
#define LX3C_LMAX_AUX 6
#define LX3C_KMAX 16

/* lx3c_dfj_plan flags */
#define LX3C_DFJ_GRADIENT 1
#define LX3C_DFJ_CONTRACT 2

typedef struct lx3c_basis lx3c_basis;
typedef struct lx3c_plan lx3c_plan;
typedef struct lx3c_dfj lx3c_dfj;
typedef struct lx3c_batch lx3c_batch;
typedef struct lx3c_metric lx3c_metric;

/* Thread-local description of the last failure in this thread. */
const char* lx3c_last_error(void);

/* Library version string. */
const char* lx3c_version(void);

/*
 * Basis (shell table) — paper Appendix A (contracted Cartesian Gaussian shells).
 *   nshell      number of shells (>= 0)
 *   l[nshell]   angular momentum per shell (host)
 *   k[nshell]   number of primitives per shell, 1..LX3C_KMAX (host)
 *   xyz[3*nshell] centres, bohr (host)
 *   atom[nshell] owning atom index (>= 0) or NULL (host); used by gradients
 *   exps, coefs  primitive exponents (> 0, finite) and coefficients, shell-major,
 *                sum(k) entries each (host)
 * Copies everything to the device; returns LX3C_EINVAL on malformed input,
 * LX3C_ENOTSUP if a shell exceeds the limits.
 */
lx3c_status lx3c_basis_create(lx3c_basis** out, int64_t nshell, const int32_t* l, const int32_t* k,
                              const double* xyz, const int32_t* atom, const double* exps,
                              const double* coefs, void* stream);
void lx3c_basis_destroy(lx3c_basis* b);

/*
 * Plan for one homogeneous integral class (la, lb | lc), paper Sec. 2.5.1.
 *   orb, aux      bases for the bra and the ket shells
 *   pairs[2*npair] host list of (a, b) shell indices into orb; all pairs must
 *                 share (l_a, k_a, l_b, k_b)
 *   auxs[naux]    host list of ket shell indices into aux; all must share (l, k)
 *   bra_pure      1: solid-harmonic bra, 0: Cartesian bra
 * Builds the class recurrence tables, uploads the lists, and allocates the
 * plan's device scratch (primitive-pair records).  Returns LX3C_EINVAL for an
 * empty or mixed list or an index out of range.
 */
lx3c_status lx3c_eri3c_plan(lx3c_plan** out, const lx3c_basis* orb, const lx3c_basis* aux,
                            const int32_t* pairs, int64_t npair, const int32_t* auxs, int64_t naux,
                            int bra_pure, void* stream);

/*
 * Evaluate the plan's integrals into out (device, npair*naux*nA*nB*nC doubles,
 * layout above).  Runs the primitive-pair precompute and the integral kernel
 * on `stream`.
 */
lx3c_status lx3c_eri3c_execute(lx3c_plan* plan, double* out, void* stream);

/* Size of one (pair, aux) block (nA*nB*nC) and the plan's total output length. */
lx3c_status lx3c_plan_sizes(const lx3c_plan* plan, int64_t* block, int64_t* total);

/*
 * Launch shape of a plan (for benchmarks and diagnostics).  Writes up to n
 * int64 values: [kernel launches per execute, then for each of the two
 * orientations (recurrences on A, on B): sub-pairs, triples per tile T,
 * primitive chunk G, lane mode, dynamic shared memory bytes, grid size;
 * then (index 13) the algorithmic flops of one execute, rounded: every
 * sub-pair's primitive pairs through its orientation's primitive stages and,
 * per ket shell, its contracted stages (a pair split across the two
 * orientations pays the contracted stages twice)].
 *
 * Orientation: a pair runs in the orientation with the smaller weighted HRR
 * amplification when that is within the threshold (lx3c_set_orientation_
 * threshold); otherwise its primitive pairs are split by compact centre.
 */
lx3c_status lx3c_plan_info(const lx3c_plan* plan, int64_t* out, int n);

void lx3c_plan_destroy(lx3c_plan* plan);

/*
 * One-call host-buffer form of lx3c_eri3c_plan + lx3c_eri3c_execute: shell
 * tables, lists and the output are host memory; device memory is allocated
 * and freed inside the call, which synchronises `stream` before returning.
 * out_host receives npair*naux*nA*nB*nC doubles (same layout as execute).
 * The output is produced in pair-range chunks of about 512 MB that alternate
 * between two device buffers; each chunk is copied to out_host on a second
 * stream while the next is computed, so the device holds two chunks, not the
 * whole output.  The two buffers (at most ~1 GB, or two pairs' blocks if
 * larger), the copy stream and its events are made on the first call and
 * kept per device for later calls; concurrent calls on one device take turns.
 * Page-locked out_host gives the full copy rate.
 */
lx3c_status lx3c_eri3c_host(int64_t orb_nshell, const int32_t* orb_l, const int32_t* orb_k,
                            const double* orb_xyz, const double* orb_exps, const double* orb_coefs,
                            int64_t aux_nshell, const int32_t* aux_l, const int32_t* aux_k,
                            const double* aux_xyz, const double* aux_exps, const double* aux_coefs,
                            const int32_t* pairs, int64_t npair, const int32_t* auxs, int64_t naux,
                            int bra_pure, double* out_host, void* stream);

/*
 * Boys function F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy (Appendix A) on the
 * device, by the same evaluator the integral kernels use (Sec. 2.5.2):
 * out[i*(mmax+1) + m] = F_m(T[i]) for m = 0..mmax, 0 <= mmax <= 24.
 * T (device, n values >= 0), out (device).
 */
lx3c_status lx3c_boys(const double* T, int64_t n, int mmax, double* out, void* stream);

/*
 * Measured FP64 FMA throughput of the current device (not in the paper; the
 * roofline denominator of the FP64-bound integral kernels): one kernel of
 * `iters` steps of an 8 x 8 register outer product per thread (64 independent
 * FMAs on 16 operands read from shared memory, as in a DGEMM), every SM
 * filled, timed with CUDA events on `stream` after a short warm-up launch.
 * *gflops = 2 * 64 * iters * threads / seconds / 1e9; *ms (may be NULL) = the
 * timed launch's duration.  Allocates and frees a small device buffer and
 * synchronises `stream`.  LX3C_EINVAL for iters < 1 or a NULL gflops.
 */
lx3c_status lx3c_fp64_rate(int64_t iters, double* gflops, double* ms, void* stream);

/*
 * Algorithmic FP64 floating-point operations (FMA = 2) for one contracted
 * (pair, aux) triple of class (la, lb | lc) with Kab primitive pairs and Kc
 * ket primitives, counted on the FLOP-minimal form of the scheme.
 */
lx3c_status lx3c_class_flops(int la, int lb, int lc, int Kab, int Kc, int bra_pure, double* flops);

/*
 * Launch-shape tuning (not in the paper).  The planner sizes a tile (triples
 * per tile T, primitive chunk G) for two CTAs per SM by default.
 * lx3c_shape_hint makes every later plan of class (la, lb | lc) -- as the
 * planner orients it, so (lb, la | lc) for the B-oriented launch -- with kab
 * primitive pairs in its largest sub-pair and kc ket primitives size its tile
 * for ctas_per_sm CTAs per SM instead (1..3; 0 removes the hint).
 * Process-wide, thread-safe; plans made before the call keep their shapes.
 * lx3c_shape_query: out[4] = {T, G, lane mode, dynamic shared memory bytes}
 * of that class for naux ket shells at ctas_per_sm CTAs per SM (0: the shape
 * the planner picks now, hints included); host only, no device needed.
 * Both return LX3C_EINVAL for arguments out of range.
 */
lx3c_status lx3c_shape_hint(int la, int lb, int lc, int bra_pure, int kab, int kc, int ctas_per_sm);
/*
 * lx3c_tile_hint fixes the tile of later plans of that class (as oriented),
 * kab and kc instead: T triples per tile (1..512) in chunks of G primitives
 * (1..kab*kc; the planner balances G over the chunks).  It takes precedence
 * over lx3c_shape_hint when the tile fits one CTA's shared memory, and is
 * ignored otherwise.  T = 0 removes it.  Process-wide, thread-safe;
 * LX3C_EINVAL for arguments out of range.
 */
lx3c_status lx3c_tile_hint(int la, int lb, int lc, int bra_pure, int kab, int kc, int T, int G);

/*
 * HRR variant of class (la, lb | lc) as the planner orients it (Sec. 2.5.5):
 * variant 0 moves one quantum per round (Eq. hrr, lb rounds with a barrier
 * each, the fewest FLOPs); variant 1 moves two per round,
 *   (a, b+1_i+1_k) = (a+1_i+1_k, b) + AB_i (a+1_k, b) + AB_k (a+1_i, b) + AB_i AB_k (a, b),
 * with one 1-q round last when lb is odd (lb/2 + lb%2 rounds, more FLOPs, no
 * first-round intermediates); -1 removes the hint (variant 0).  Read by later
 * plans; process-wide, thread-safe.  LX3C_EINVAL for arguments out of range.
 */
lx3c_status lx3c_hrr_hint(int la, int lb, int lc, int bra_pure, int variant);
/* Host self-check of that variant's tables (no device needed): the table
 * invariants of lx3c_class_tables_check, then the HRR rows applied to moment
 * integrals int (x-A)^a (x-B)^b w(x) dx, for which Eq. hrr is exact;
 * *max_rel_err = the largest error against their closed form relative to
 * the sum of its term magnitudes. */
lx3c_status lx3c_hrr_tables_check(int la, int lb, int lc, int bra_pure, int variant, const double* AB,
                                  double* max_rel_err);

/*
 * Accuracy settings (not in the paper), process-wide and thread-safe, read
 * by every later plan (plans made before the call keep theirs):
 * lx3c_set_orientation_threshold: HRR (Eq. hrr) moves the recurrence centre's
 *   quanta to the other centre through AB; when P sits close to the target
 *   centre this cancels and amplifies FP64 rounding.  A pair keeps one
 *   orientation when its worst weighted amplification estimate there is at
 *   most amp_max, otherwise each primitive pair runs its recurrences on its
 *   more compact centre (a second, transposed launch).  Smaller values split
 *   more pairs (more accurate, more post-contraction work).  amp_max >= 1,
 *   or 0 for the default 300; else LX3C_EINVAL.
 * lx3c_set_compensation: bits selecting compensated (Dot2: TwoProduct by FMA
 *   and TwoSum) summation in the contracted stages -- bit 0 the n-quantum
 *   CVRR2 gather (Sec. 2.5.4), bit 1 the ket Cartesian-to-solid-harmonic
 *   transform; 0 (the default) for plain FMA chains.  bits outside 0..3 give
 *   LX3C_EINVAL.
 */
lx3c_status lx3c_set_orientation_threshold(double amp_max);
lx3c_status lx3c_set_compensation(int bits);

/*
 * Self-check of the planner's host tables for class (la, lb | lc) (not in the
 * paper): every VRR1 (Eq. vrr1) item reads only entries formed at lower
 * levels and every entry above level 0 is formed exactly once; weight,
 * accumulator, gather (Sec. 2.5.4), ket/bra transform and HRR (Eq. hrr)
 * indices are in range; HRR level j reads only level j-1; the gather order is
 * a permutation by descending term count and its sliced-ELL copy holds the
 * CSR terms, padded with zero-coefficient terms.  Host only.  Returns LX3C_OK,
 * or LX3C_EINVAL naming the first violation (lx3c_last_error).
 */
lx3c_status lx3c_class_tables_check(int la, int lb, int lc, int bra_pure);
lx3c_status lx3c_shape_query(int la, int lb, int lc, int bra_pure, int kab, int kc, int64_t naux, int ctas_per_sm,
                             int32_t* out);

/* Library's solid-harmonic matrix for shell l: out[(m+l)*ncart(l) + c]. */
lx3c_status lx3c_solid_harmonics(int l, double* out);

/*
 * n-quantum CVRR2 expansion (Sec. 2.5.4) of the contracted target (a 0|c)
 * as the library tabulates it: for bra exponents a[3], ket exponents c[3]
 * writes up to cap terms (e[3], k, n[3], coef) into terms[8*i..8*i+7] as
 * doubles and their count into *nterms.
 */
lx3c_status lx3c_cvrr2_expansion(const int32_t* a, const int32_t* c, int32_t cap, double* terms,
                                 int32_t* nterms);

/*
 * Density-fitted Coulomb build (paper Sec. 3: the DF-J builder fed by an
 * integral-digestion callable; integrals never reach global memory):
 *   gamma_P = sum_{mu nu} (mu nu|P) D_{mu nu},   J_{mu nu} = sum_P (mu nu|P) c_P
 * over all AO pairs of the orbital basis (all shells solid harmonic, AO order =
 * shell order, components m = -l..l), for every ket shell P of the aux basis.
 *
 * lx3c_dfj_plan: setup (synchronises `stream`, not part of the timed path).
 *   flags LX3C_DFJ_GRADIENT (bit 0): also prepare the nuclear gradient
 *   (lx3c_dfj_grad); needs an atom index on every shell and orbital shells
 *   with l < LX3C_LMAX_ORB.
 *   flags LX3C_DFJ_CONTRACT (bit 1): digest at the (e 0|c) level, the DF-J
 *   analogue of the J-engine the paper names as the follow-up (Sec. 4: the
 *   density is contracted with integral intermediates rather than with the
 *   integrals): per pair launch the bra map M (the HRR and bra transforms,
 *   (AB|C) = sum_e M[AB][e] (e 0|C)) is formed once per pair; per triple
 *   gamma_P = sum_c T_Cc sum_e (M^T D)_e (e 0|c) and y_e += sum_c (e 0|c)
 *   (T^T c_P)_c, then J_AB += M y per pair -- no ket transform, HRR or bra
 *   transform per triple.  A launch keeps the per-integral digestion when its
 *   bra map does not fit in shared memory, or when the contracted form would
 *   take more flops (few kets per pair: the per-pair bra maps cost more than
 *   the per-triple stages they replace).  Same results to rounding.
 *   Screening: a (pair, ket) triple is kept when Q_ab Q_P >= schwarz_tol, with
 *   Q_ab = 20 sum over primitive pairs of |c_a c_b| exp(-za zb/g AB^2)
 *   sqrt(2 pi^{5/2}/(g^2 sqrt(2g))) (|PA|^2+1/(2g))^{la/2} (|PB|^2+1/(2g))^{lb/2}
 *   and Q_P = sum |c_c| sqrt(2 pi^{5/2}/(z^2 sqrt(2z))) (1/(2z))^{lc/2}: 20x an
 *   analytic estimate of sqrt(max|(ab|ab)|) sqrt(max|(P|P)|), which is not a
 *   bound by itself (the largest element of a triple reaches ~11x the
 *   unscaled estimate on the DF-J recipe's clusters); the factor 20 keeps the
 *   dropped integrals below schwarz_tol there (lx3c_schwarz_pair/aux return
 *   the library's Q values).  Pass 0 to keep all.
 *   Returns LX3C_ENOTSUP for orbital shells above LX3C_LMAX_ORB.
 * lx3c_dfj_execute: D (device, nao x nao row-major, symmetric), c (device,
 *   naux_ao) in; gamma (device, naux_ao) and J (device, nao x nao, symmetric)
 *   overwritten; either output may be NULL to skip it (not both).
 *   Asynchronous on `stream`.  gamma and J are summed exactly in fixed point
 *   (each contribution rounded to a multiple of 2^-72, every partial sum
 *   below 2^55 in magnitude) and rounded once to FP64, so the
 *   result does not depend on the order in which tiles finish: repeated
 *   executes of a plan are bitwise equal.
 * lx3c_dfj_execute_multi: the same build for nd (1..8) densities and
 *   coefficient vectors at once, sharing every integral: D (device, nd x nao
 *   x nao), c (device, nd x naux_ao) in; gamma (nd x naux_ao) and J (nd x nao
 *   x nao) overwritten, either may be NULL to skip it (then its input may be
 *   NULL too).  Per tile the digestion is two small GEMMs (gamma: (tile kets x
 *   components) x (pair block) times (pair block) x nd; J: (pair block) x
 *   (tile kets x components) times that x nd) on FP64 tensor-core tiles
 *   (mma.sync m8n8k4), nd zero-padded to 8; gamma and J are summed with
 *   FP64 atomics here (order-dependent in the last bits).  LX3C_ENOTSUP if a
 *   class's scratch does not fit.  Asynchronous.
 * lx3c_dfj_energy: gamma as above (J skipped) and *energy = c^T gamma
 *   (device scalar), the DF-J energy whose gradient lx3c_dfj_grad returns.
 * lx3c_dfj_info: out[0..10] = groups, screened (pair, ket shell) triples,
 *   integrals digested, algorithmic FP64 flops per execute, kernel launches
 *   per execute, nao, naux_ao, natom, gradient FP64 flops, gradient launches,
 *   tile slots of the integral launches (screened triples / slots is the
 *   tile fill).
 * lx3c_dfj_grad: dE/dR for E = c^T gamma with D and c held fixed (not in the
 *   paper): for every screened triple the derivative integrals
 *   d/dA (ab|P) = sum_prim [2 za (a+1 b|P) - a (a-1 b|P)] (same for B) are
 *   formed on the fly in Cartesian-bra classes and contracted with
 *   W = w D_ab c_P; dE/dC = -(dE/dA + dE/dB) (translational invariance).
 *   grad (device, natom x 3) overwritten; summed in the same exact fixed
 *   point as gamma and J (bitwise reproducible).
 * lx3c_dfj_group: the screened task list of class group gi (for checks):
 *   info[8] = {la, lb, lc, ka, kb, kc, npair, nket}; pairs[2*npair] shell
 *   indices (a, b); counts[npair]: pair i is kept with the first counts[i]
 *   entries of auxs[nket] (ket shells sorted by decreasing Q_P).  Any output
 *   pointer may be NULL.
 */
lx3c_status lx3c_dfj_plan(lx3c_dfj** out, const lx3c_basis* orb, const lx3c_basis* aux, double schwarz_tol,
                          int flags, void* stream);
/* The screening factors Q_ab (with the factor 20) and Q_P of lx3c_dfj_plan for
 * one shell pair (l, K, centre[3], exponents[K], coefficients[K] per shell)
 * or one ket shell; host only, no device needed.  LX3C_EINVAL on NULL or
 * l < 0, K < 1. */
lx3c_status lx3c_schwarz_pair(int la, int ka, const double* A, const double* ea, const double* ca, int lb, int kb,
                              const double* B, const double* eb, const double* cb, double* q);
lx3c_status lx3c_schwarz_aux(int l, int k, const double* e, const double* c, double* q);
lx3c_status lx3c_dfj_execute(lx3c_dfj* plan, const double* D, const double* c, double* gamma, double* J,
                             void* stream);
lx3c_status lx3c_dfj_execute_multi(lx3c_dfj* plan, int nd, const double* D, const double* c, double* gamma,
                                   double* J, void* stream);
lx3c_status lx3c_dfj_energy(lx3c_dfj* plan, const double* D, const double* c, double* gamma, double* energy,
                            void* stream);

/*
 * Tile-callback DF-J build (paper Sec. 3: the DF-J builder's end-user
 * interface receives tiles of the density matrix and writes tiles of J
 * through callables, assuming nothing about their layout or distribution).
 * The orbital AOs are cut into consecutive blocks of whole shells of about
 * tile_ao AOs each; a tile is (row block, column block).
 *   get_D(user, row0, nrow, col0, ncol, dst, ld): fill the host buffer dst
 *     (nrow x ncol, row stride ld) with D[row0.., col0..]; asked for the
 *     tiles with row block <= column block only (D must be symmetric).
 *   put_J(user, row0, nrow, col0, ncol, src, ld): take J[row0.., col0..]
 *     from the host buffer src (valid during the call only); called for every
 *     tile, row-block-major, after the build.  May be NULL (gamma only).
 *   Either callable returns 0 on success; any other value stops the build
 *   with LX3C_EINVAL.
 *   c (host, naux_ao) in; gamma (host, naux_ao) out, may be NULL.
 * Device copies of D and J and two page-locked staging tiles are allocated
 * and freed inside the call, which synchronises `stream`.  The callables run
 * on the calling thread.
 */
typedef int (*lx3c_tile_get_fn)(void* user, int64_t row0, int64_t nrow, int64_t col0, int64_t ncol, double* dst,
                                int64_t ld);
typedef int (*lx3c_tile_put_fn)(void* user, int64_t row0, int64_t nrow, int64_t col0, int64_t ncol,
                                const double* src, int64_t ld);
lx3c_status lx3c_dfj_execute_tiles(lx3c_dfj* plan, int64_t tile_ao, lx3c_tile_get_fn get_D,
                                   lx3c_tile_put_fn put_J, void* user, const double* c, double* gamma,
                                   void* stream);
lx3c_status lx3c_dfj_grad(lx3c_dfj* plan, const double* D, const double* c, double* grad, void* stream);
lx3c_status lx3c_dfj_info(const lx3c_dfj* plan, double* out, int n);
lx3c_status lx3c_dfj_group(const lx3c_dfj* plan, int gi, int32_t* info, int32_t* pairs, int32_t* counts,
                           int32_t* auxs);
void lx3c_dfj_destroy(lx3c_dfj* plan);

/*
 * Density-fitting metric and solve.  The paper's DF-J (Sec. 1: density
 * fitting of the Coulomb operator; Sec. 4: DF-J with a J-fitting auxiliary
 * basis) fits the density as c = V^{-1} gamma with the Coulomb metric
 * V_PQ = (P|Q) of the auxiliary basis, then forms J_{mu nu} = sum_P (mu nu|P) c_P.
 *
 * lx3c_metric_plan: plan V for an aux basis (all shells, any mix of l <=
 *   LX3C_LMAX_AUX and K).  (P|Q) is evaluated by the class kernels as the
 *   3-centre integral (P 1|Q) whose second bra function is the constant 1
 *   (an s Gaussian with exponent 0), one (l_P 0 | l_Q) class launch per pair
 *   of (l, K) shell groups.  Setup; synchronises `stream`.
 * lx3c_metric_execute: V (device, naux_ao x naux_ao row-major, AO order =
 *   shell order, components m = -l..l) receives every element, both
 *   triangles (V is symmetric).  Asynchronous on `stream`.
 * lx3c_metric_info: out[0..5] = naux_ao, shell groups, class launches,
 *   kernel launches per execute, algorithmic FP64 flops per execute, shell
 *   pairs.
 * lx3c_cholesky: in-place Cholesky V = L L^T of the symmetric positive
 *   definite A (device, n x n row-major, leading dimension lda >= n), reading
 *   and writing only the lower triangle (the strictly upper triangle is left
 *   as it was).  Blocked right-looking, 64-wide panels, FP64 throughout.
 *   info (device int32, may be NULL) is set to 0, or to the 1-based index of
 *   the first non-positive pivot (the factor then holds NaN from there on).
 *   drop_tol = 0: info gets the first non-positive pivot as above.
 *   drop_tol in (0, 1): a pivot at or below drop_tol times A's original
 *   diagonal element marks that function as linearly dependent on the
 *   earlier ones (the usual treatment of a near-singular fitting metric):
 *   its diagonal entry becomes +inf and its column below the diagonal 0, so
 *   lx3c_cholesky_solve gives it a zero coefficient; info gets the number of
 *   functions dropped.  This mode takes n doubles of stream-ordered scratch
 *   (cudaMallocAsync).
 *   Asynchronous on `stream`; LX3C_EINVAL for n < 1, lda < n, a NULL A or
 *   drop_tol outside [0, 1).
 * lx3c_cholesky_solve: B <- (L L^T)^{-1} B with L from lx3c_cholesky and B
 *   (device, n x nrhs row-major, the nrhs right-hand sides contiguous per
 *   row) overwritten.  Asynchronous on `stream`.
 * lx3c_dfj_coulomb: the whole DF-J Coulomb build from a DF-J plan (screened
 *   integrals, lx3c_dfj_plan) and the metric's Cholesky factor L (lda >=
 *   naux_ao): gamma = sum (mu nu|P) D_{mu nu} (device, naux_ao out),
 *   c = V^{-1} gamma (device, naux_ao out), J = sum_P (mu nu|P) c_P (device,
 *   nao x nao out).  Two integral passes and one solve; asynchronous.
 */
lx3c_status lx3c_metric_plan(lx3c_metric** out, const lx3c_basis* aux, void* stream);
lx3c_status lx3c_metric_execute(lx3c_metric* plan, double* V, void* stream);
lx3c_status lx3c_metric_info(const lx3c_metric* plan, double* out, int n);
void lx3c_metric_destroy(lx3c_metric* plan);
lx3c_status lx3c_cholesky(double* A, int64_t n, int64_t lda, double drop_tol, int32_t* info, void* stream);
lx3c_status lx3c_cholesky_solve(const double* L, int64_t n, int64_t lda, double* B, int64_t nrhs, void* stream);
lx3c_status lx3c_dfj_coulomb(lx3c_dfj* plan, const double* L, int64_t lda, const double* D, double* gamma,
                             double* c, double* J, void* stream);

/*
 * Batched uneven workload (not in the paper; the paper launches one class per
 * kernel): DF-J builds of several molecules, every class mixed, run from one
 * CUDA graph launch.
 *
 * lx3c_batch_plan: one DF-J plan per molecule (orbs[m], auxs[m], screening as
 *   in lx3c_dfj_plan), then an autotuner picks the triples-per-tile shape of
 *   every launch signature (class, orientation, contraction, Kc) by timing
 *   candidates on a fixed prefix (about eight waves of tiles) of the
 *   signature's largest launch; results are read from and written to the
 *   text file tune_cache ("key T" lines) when it is non-NULL.  Setup;
 *   synchronises `stream`.
 * lx3c_batch_bind: fixes the per-molecule device buffers (D[m] nao x nao,
 *   c[m] naux_ao in; gamma[m], J[m] out; all owned by the caller and kept
 *   alive while the batch is executed), orders the class launches longest
 *   first and captures two CUDA graphs of the whole build (zeroing,
 *   precompute, integrals, J finish): graph 1 runs every (class launch,
 *   tile) work item in persistent kernels, one per occupancy tier (the
 *   items that fit three CTAs per SM of the 40-register persistent kernel,
 *   then two CTAs of the unrestricted one, then the rest), each sized for its
 *   tier's largest item and pulling items longest first from its own atomic
 *   counter (no CTA waits on another); graph 2 runs the class launches
 *   themselves on four parallel graph branches.  Setup; may
 *   synchronise.  Returns LX3C_ECUDA if a capture fails.
 * lx3c_batch_execute: mode 1 or 2 launches graph 1 or 2 (one
 *   cudaGraphLaunch on `stream`); mode 0 runs the same tasks as per-class
 *   launches (lx3c_dfj_execute per molecule), for comparison; any other mode
 *   is LX3C_EINVAL.  Asynchronous.  Modes 0 and 2 run the same kernels and
 *   give bitwise equal results; mode 1's persistent kernels run the tile form
 *   for every class ((s s|C) included, which the class launches run
 *   register-resident), so mode 1 agrees with them to rounding.
 * lx3c_batch_info: out[0..15] = molecules, screened triples, integrals,
 *   algorithmic flops, plain kernel launches, persistent-graph kernel nodes,
 *   work items, class launches merged, persistent smem bytes, persistent
 *   grid, tuned signatures, signatures measured by this plan, branch-graph
 *   kernel nodes, branches, tile slots (tiles x triples per tile, summed
 *   over launches; screened triples / slots is the tile fill), persistent
 *   tiers.  (out[0..15].)
 */
lx3c_status lx3c_batch_plan(lx3c_batch** out, int nmol, const lx3c_basis* const* orbs,
                            const lx3c_basis* const* auxs, double schwarz_tol, const char* tune_cache,
                            void* stream);
lx3c_status lx3c_batch_bind(lx3c_batch* batch, const double* const* D, const double* const* c,
                            double* const* gamma, double* const* J, void* stream);
lx3c_status lx3c_batch_execute(lx3c_batch* batch, int mode, void* stream);
lx3c_status lx3c_batch_info(const lx3c_batch* batch, double* out, int n);
void lx3c_batch_destroy(lx3c_batch* batch);

/*
 * Allocation-free form of one (la lb|lc) class evaluation.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory
 * around the call -- for example code that runs while a memory pool owns the
 * device heap (a raw cudaMalloc then fails or fragments the pool) or code that
 * must not stall the device (cudaFree synchronises the whole device).
 *
 * Inputs and the output are the caller's, all device pointers:
 *   la, lb, lc, ka, kb, kc  the class and contraction degrees; every pair in
 *                           `pairs` must have an l=la, k=ka first shell and an
 *                           l=lb, k=kb second shell, every ket shell in `auxs`
 *                           l=lc, k=kc (not checked: the lists stay on the device)
 *   *_off, *_xyz, *_exps, *_coefs  shell tables as in lx3c_basis_create
 *                           (off[s] = index of shell s's first primitive)
 *   pairs[2*npair], auxs[naux]  shell indices; out: npair*naux*nA*nB*nC
 *                           doubles, same layout as lx3c_eri3c_execute.
 * Everything else the path needs (primitive records, sub-pair lists, Boys
 * and index tables) lives in one statically sized device array of about
 * 27 MB that every GPU loading the library holds until process exit.
 * Limits: npair <= 65536, npair*ka*kb <= 65536, naux*kc <= 65536; larger
 * problems are rejected with LX3C_ENOTSUP and nothing is launched.
 * First call on a device (once per process and device): it looks up the
 * array's device address, builds the Boys table on the host and copies it and
 * the constant tables in with synchronous copies (cudaMemcpy,
 * cudaMemcpyToSymbol), which wait for the device.  Make that first call before
 * any stream capture begins.
 * Every call: the class's index tables (both orientations, at most 4 MB, held
 * in host memory the library keeps for the process) are copied into the array
 * by cudaMemcpyAsync from pageable host memory.  CUDA stages such a copy
 * through a buffer of its own, so the call can return only after the copy is
 * staged and may first wait for work already queued on `stream`; the
 * precompute and integral kernels are then queued on `stream` and the call
 * returns without waiting for them.
 * All calls share the array and each overwrites it: calls that overlap on the
 * GPU (for instance on different streams) race; calls on one stream are
 * ordered.  No device memory is allocated or freed, on any call.
 */
lx3c_status lx3c_eri3c_noalloc(int la, int lb, int lc, int ka, int kb, int kc, int bra_pure,
                               const int64_t* orb_off, const double* orb_xyz, const double* orb_exps,
                               const double* orb_coefs, const int64_t* aux_off, const double* aux_xyz,
                               const double* aux_exps, const double* aux_coefs, const int32_t* pairs,
                               int64_t npair, const int32_t* auxs, int64_t naux, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LX3C_H */
