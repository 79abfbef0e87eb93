/*
 * goac.h -- C ABI of the GB300 (sm_103a) library for the pairwise Coulomb
 * cluster-expansion optimiser of "Optimization of Coulomb Energies in
 * Gigantic Configurational Spaces of Multi-Element Ionic Crystals" (GOAC).
 *
 * Conventions (apply to every entry point):
 *  - Pointers named *_dev are device pointers on the context's device, owned
 *    by the caller; *_host pointers are host memory owned by the caller.
 *    Shapes are row-major; "B x Nv" means B rows of Nv contiguous entries.
 *  - Work is enqueued on the context's CUDA stream and is stream-ordered.
 *    Calls that say "synchronises" block until their work is finished.
 *  - The library allocates only its own scratch memory (owned by a context or
 *    a problem, freed by the matching destroy call).
 *  - Every call returns a goac_status; on failure goac_last_error() gives a
 *    message (thread-local).  No C++ exception crosses the ABI.
 *  - Empty batches: a call whose number of configurations, chains or
 *    individuals (B, C, P, G) is 0 does nothing and returns GOAC_OK; its
 *    per-configuration buffers may then be NULL (the problem or context
 *    handle is still required, and the other arguments are still checked).
 *    A negative count, or one above GOAC_MAX_BATCH, is GOAC_ERR_INVALID_ARG.
 *  - Bounded waits: no kernel of this library waits without an iteration
 *    limit; a wait that runs out sets a device error word that the next
 *    synchronising call reports as GOAC_ERR_TIMEOUT.
 *  - Problems: N sites; site_class[i] = -1 marks a fixed ion of charge
 *    fixed_q[i], otherwise the index (0..n_class-1) of the partially
 *    occupied site class the position belongs to (the paper's "site" with
 *    P_s positions, Eq. 1).  S species with charges z[s]; counts[k*S + s] is
 *    the number of ions of species s in class k (the occupancies O_i of
 *    Eq. 2c1; 0 = species not allowed in that class).  A configuration is one
 *    int8 species index per variable site, variable sites in ascending site
 *    order (Nv of them), which satisfies Eq. 2c2/2c3 by construction.
 *  - Energies in eV, lengths in Angstrom, kT in eV.
 */
#ifndef GOAC_H
#define GOAC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t goac_status;

#define GOAC_OK 0
#define GOAC_ERR_INVALID_ARG (-1)   /* bad sizes, pointers, counts             */
#define GOAC_ERR_CUDA (-2)          /* a CUDA runtime/driver call failed        */
#define GOAC_ERR_OOM (-3)           /* scratch allocation failed                */
#define GOAC_ERR_NOT_NEUTRAL (-4)   /* total charge |sum q| > 1e-9              */
#define GOAC_ERR_TIMEOUT (-5)       /* a bounded device wait ran out            */
#define GOAC_ERR_INTERNAL (-6)      /* device-side consistency check failed     */
#define GOAC_ERR_UNSUPPORTED (-7)   /* device is not sm_103 / feature missing   */

/* Largest number of configurations, chains or individuals in one call:     *
 * 2^31 - 256, so that a batch padded to whole 256-configuration tiles still *
 * has an int32 count.                                                       */
#define GOAC_MAX_BATCH 2147483392

/* Arithmetic forms of the batched scoring E = q^T J q. */
#define GOAC_PREC_F64 0     /* FP64 CUDA-core GEMM: the plain path              */
#define GOAC_PREC_TF32 1    /* tcgen05 kind::tf32, J rounded to TF32, 1 term     */
#define GOAC_PREC_TF32X2 2  /* tcgen05 kind::tf32, J = hi + lo (TF32 each)       */
#define GOAC_PREC_BF16X2 3  /* tcgen05 kind::f16 (BF16), J = J1 + J2             */
#define GOAC_PREC_BF16X3 4  /* tcgen05 kind::f16 (BF16), J = J1 + J2 + J3        */
#define GOAC_PREC_F32 5     /* FP32 CUDA cores (Monte Carlo / GA variant only)   */
#define GOAC_PREC_EXACT 6   /* tcgen05 integer-digit split (FP64-grade, see below) */
#define GOAC_PREC_F64_INCR 7 /* GA runs only: incremental FP64 rescoring (goac_ga_run) */
#define GOAC_PREC_F16X2 8   /* relaxed gradient only: tcgen05 kind::f16 (FP16), J = hi + lo */

typedef struct goac_ctx goac_ctx;
typedef struct goac_problem goac_problem;

/* Last error message of the calling thread ("" if none).  Never NULL. */
const char* goac_last_error(void);

/* ABI version (major * 100 + minor). */
int32_t goac_version(void);

/* Create a context on `device` that enqueues on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Fails with GOAC_ERR_UNSUPPORTED unless
 * the device is compute capability 10.3 (GB300). */
goac_status goac_ctx_create(int32_t device, void* stream, goac_ctx** out);
goac_status goac_ctx_destroy(goac_ctx* ctx);
goac_status goac_ctx_set_stream(goac_ctx* ctx, void* stream);
/* Synchronise the context stream and report any device error word. */
goac_status goac_ctx_synchronize(goac_ctx* ctx);
/* Per-kernel timing: when enabled, a CUDA event pair is recorded on the      *
 * context stream around every launch of the timed kernel families:           *
 * 0 = tensor-core scoring, 1 = CUDA-core scoring GEMM, 2 = Monte Carlo,      *
 * 3 = GA children, 4 = Ewald real space, 5 = Ewald reciprocal SYRK,          *
 * 6 = incremental GA rescoring.                                               */
goac_status goac_ctx_set_timing(goac_ctx* ctx, int32_t enable);
/* Total recorded milliseconds and launch count of kernel family `kernel`     *
 * since the last query (waits for the recorded events; clears the record).  */
goac_status goac_ctx_kernel_time(goac_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches);
/* Failure-detection self test (no counterpart in the paper): one thread      *
 * waits on a device barrier that nothing completes, with the clock-bounded    *
 * wait every waiting kernel of this library uses (limit_cycles SM cycles,     *
 * 1 .. 4e9).  Returns GOAC_ERR_TIMEOUT once the wait has run out; the context *
 * remains usable.  Synchronises.                                              */
goac_status goac_selftest_wait_timeout(goac_ctx* ctx, int64_t limit_cycles);
/* Number of kernels this library has launched in the process so far. */
int64_t goac_launch_count(void);

/* ------------------------------------------------------------------------ *
 * Ewald pair matrix J (Section "Cluster Expansion of Coulomb Energy": the  *
 * second-order expansion is exact for point charges; its coefficients are  *
 * Ewald energies).  With q the charges of all N sites, E = q^T J q where    *
 *   J_ij = ke/2 [ sum'_n erfc(alpha|d+n|)/|d+n|                             *
 *               + (4 pi/V) sum_{0<|k|<=kcut} exp(-k^2/4alpha^2)/k^2 cos(k.d)*
 *               - (2 alpha/sqrt(pi)) delta_ij - pi/(V alpha^2) ],           *
 * d = minimum-image r_j - r_i (fractional components wrapped to [-1/2,1/2)),*
 * n over lattice translations |n_a| <= nimg[a] (n = 0 dropped for i == j),  *
 * k over reciprocal vectors with |k| <= kcut (both k and -k).  Real-space   *
 * terms with alpha|d+n| >= 8 (erfc < 1.2e-29) are skipped.                  *
 *   lattice_host: 3x3 row-major, rows = lattice vectors (Angstrom).         *
 *   frac_dev: N x 3 fractional coordinates.  ke: e^2/(4 pi eps0) in eV*A.   *
 *   J_dev: N x N FP64 output (row-major, exactly symmetric).                *
 * Synchronises (sizes of the reciprocal set are read back).                 *
 * ------------------------------------------------------------------------ */
goac_status goac_build_ewald(goac_ctx* ctx, const double* lattice_host, const double* frac_dev, int32_t N,
                             double alpha, const int32_t* nimg_host, double kcut, double ke, double* J_dev);

/* ------------------------------------------------------------------------ *
 * Problem (Eq. 2 with its constraints).  Copies what it needs from J_dev:   *
 * J_vv (variable-variable block), its diagonal, phi_fix = J_vf q_f and      *
 * E_const = q_f^T J_ff q_f (the paper's zero-order term and the fixed-ion   *
 * share of the first-order term), so that                                   *
 *   E = q_v^T J_vv q_v + 2 q_v . phi_fix + E_const.                         *
 * All array arguments except J_dev are host arrays.  Checks that every      *
 * class's counts add up to its size and that the total charge is neutral   *
 * (|sum q| <= 1e-9, else GOAC_ERR_NOT_NEUTRAL unless allow_charged != 0).   *
 * Synchronises.                                                             *
 * ------------------------------------------------------------------------ */
goac_status goac_problem_create(goac_ctx* ctx, const double* J_dev, int32_t N, const int32_t* site_class_host,
                                const double* fixed_q_host, const double* z_host, int32_t S,
                                const int32_t* counts_host, int32_t n_class, int32_t allow_charged,
                                goac_problem** out);
goac_status goac_problem_destroy(goac_problem* prob);
/* Nv and E_const of a problem (host outputs; either may be NULL). */
goac_status goac_problem_info(const goac_problem* prob, int32_t* Nv, double* E_const);
/* Copy phi_fix (Nv doubles) to a device buffer. */
goac_status goac_problem_phi_fix(const goac_problem* prob, double* phi_fix_dev);

/* ------------------------------------------------------------------------ *
 * Batched scoring of a population (Eq. 2 objective, one energy per config): *
 *   E_b = q_b^T J_vv q_b + 2 q_b . phi_fix + E_const.                       *
 *   species_dev: B x Nv int8.  E_dev: B doubles.  precision: GOAC_PREC_*.   *
 * F64 is the plain path; the tensor-core forms split J into TF32 / BF16     *
 * terms, accumulate J.Q in FP32 on tcgen05 and form E in FP64.  EXACT      *
 * (charges integers after a power-of-two scaling 2^kq, kq <= 4, and          *
 * 128 max|q 2^kq| Nv_pad < 2^24, Nv_pad = Nv rounded up to 128; else        *
 * GOAC_ERR_UNSUPPORTED): each 128-row panel of J is scaled by a power of    *
 * two and cut into T signed r-bit digits held in FP16 (r = 10, T = 5 when   *
 * 512 max|q 2^kq| Nv_pad < 2^24, else r = 8, T = 6), so every tensor-core    *
 * product and partial sum is an integer below 2^24 and exact; digit sums are *
 * weighted by the charges in 32-bit integers and combined in FP64          *
 * (truncation 2^-rT <= 2^-48 of the panel's largest entry).                 *
 * ------------------------------------------------------------------------ */
goac_status goac_score(goac_problem* prob, const int8_t* species_dev, int32_t B, int32_t precision, double* E_dev);

/* Tile shape of the tensor-core scoring kernels (no counterpart in the       *
 * paper; the results of EXACT do not depend on it, those of the split forms  *
 * change only by FP32 rounding).  A tile covers tile_m sites x tile_n        *
 * configurations: tile_m 128 (one CTA) or 256 (every form with tile_n 256:   *
 * a pair of CTAs on one TPC issuing M = 256 tcgen05 MMAs over the            *
 * configurations, each CTA loading its own 128 configurations and its own    *
 * panel's rows of J', each epilogue thread weighting one configuration's 256 *
 * site sums by its charges; EXACT only, with tile_n 128: one CTA with the    *
 * configurations on the tensor-memory lanes), tile_n 128 or 256;             *
 * ksplit > 0 cuts each row panel's column range into chunks of ksplit         *
 * 128-column blocks scored as separate tiles (the row-dot is linear, so each  *
 * chunk adds a partial sum; this spreads small populations over all SMs).    *
 * goac_score_set_shape stores a shape for (precision, B rounded up to 256)    *
 * (all 0: the default, whole ranges in 256 x 256 tiles on CTA pairs for EXACT *
 * and the BF16 forms, 128 x 256 tiles for the TF32 forms);                    *
 * goac_score_autotune times                                                   *
 * every shape in {128 x 256, 128 x 128, 256 x 256, 256 x 128 (EXACT)} x     *
 * {0, 16, 8, 4, 2}                                                            *
 * on species_dev (B x Nv), CUDA events on the context stream, stores the      *
 * fastest for later goac_score calls with that precision and padded B, and    *
 * returns it (outputs nullable; ms per scoring call).  Host-side store;       *
 * autotune synchronises.                                                      */
goac_status goac_score_set_shape(goac_problem* prob, int32_t precision, int32_t B, int32_t tile_m, int32_t tile_n,
                                 int32_t ksplit);
goac_status goac_score_autotune(goac_problem* prob, const int8_t* species_dev, int32_t B, int32_t precision,
                                int32_t* tile_m_out, int32_t* tile_n_out, int32_t* ksplit_out, double* ms_out);

/* Digit layout the EXACT form uses on this problem (host outputs, nullable):  *
 * digit_bits r, digits T and the charge scaling kq of the rule above; the     *
 * truncation of J is then at most 2^-rT of each panel's largest entry.       *
 * GOAC_ERR_UNSUPPORTED when the charges do not admit the exact form.          */
goac_status goac_problem_exact_info(const goac_problem* prob, int32_t* digit_bits, int32_t* digits,
                                    int32_t* charge_shift);

/* Allocation-free FP64 scoring, for callers that may not allocate device     *
 * memory themselves (their device memory comes from a host framework's own   *
 * pool, or they run under a no-allocation policy after start-up).  The paper *
 * has no counterpart: it is an interface variant of goac_score(F64) on raw    *
 * buffers, with no context or problem handle.  Allocates nothing: besides the *
 * caller's buffers it uses one fixed file-scope device array of 524,288        *
 * doubles (4 MiB, present on every GPU that loads the library until exit) for *
 * the per-tile partial energies; requires ceil(Nv/64) * B <= 524,288, else    *
 * GOAC_ERR_INVALID_ARG.  Each call outside a stream capture looks up that     *
 * array's device address (cudaGetSymbolAddress) and caches it per device, so  *
 * a device whose context was reset gets the new address; a call inside a      *
 * capture uses the cached one, so make a first call on each device before any *
 * stream capture (else GOAC_ERR_INVALID_ARG).  All calls share the array and  *
 * it keeps the last call's contents (every entry read is first written,      *
 * nothing needs clearing); calls that overlap on the GPU race on it.         *
 *   Jvv_dev: ceil(Nv/64)*64 rows of `ld` doubles (ld >= Nv rounded up to 64),  *
 *            J_vv in the leading Nv x Nv block, finite values elsewhere.      *
 *   species_dev: B x Nv int8, every value in 0 .. 63 (it indexes z_dev; a     *
 *   value outside is not checked and gives undefined energies).  z_dev: 64    *
 *   doubles (charges of species 0..S-1, any finite values after).             *
 *   phi_fix_dev: ld doubles (phi_fix in the first Nv, zeros when there are    *
 *   no fixed ions).  E = q^T J_vv q + 2 q . phi_fix + E_const into E_dev      *
 *   (B doubles).  Runs on the current device, on `stream`.                    */
goac_status goac_score_f64_noalloc(const double* Jvv_dev, int32_t ld, int32_t Nv, const int8_t* species_dev,
                                   int32_t B, const double* z_dev, const double* phi_fix_dev, double E_const,
                                   void* stream, double* E_dev);

/* Same, with host buffers: copies species H2D, scores, copies E D2H on the  *
 * context stream and synchronises (end-to-end entry point).                 */
goac_status goac_score_host(goac_problem* prob, const int8_t* species_host, int32_t B, int32_t precision,
                            double* E_host);

/* Pipelined host-buffer scoring for a stream of populations (the paper's    *
 * objective, Eq. 2, as in goac_score; the paper has no counterpart: its     *
 * populations live in host memory next to its CPU code).  Enqueues, without *
 * waiting: the H2D copy of species_host (B x Nv int8) into one of two        *
 * device staging slots on the context's own copy stream, the scoring on the *
 * context stream once that copy has landed, and the D2H copy of the B       *
 * energies into E_host.  Consecutive calls alternate slots, so the copy of  *
 * call k+1 overlaps the scoring of call k; a slot is refilled only after    *
 * the scoring that read it has finished.  The caller keeps species_host     *
 * unchanged and does not read E_host until goac_ctx_synchronize(ctx)        *
 * returns.  Both host buffers should be page-locked: with pageable memory   *
 * the copies are correct but block the host, and nothing overlaps.  Errors  *
 * of the enqueued work are reported by goac_ctx_synchronize.                */
goac_status goac_score_host_async(goac_problem* prob, const int8_t* species_host, int32_t B, int32_t precision,
                                  double* E_host);

/* Top-k "n lowest structures" (Section "Implementation and Theoretical      *
 * Background": the n lowest configurations are the output).  Selects the k  *
 * lowest E_approx (ties: lower index), rescores them in FP64 and returns     *
 * them sorted by the FP64 energy (ties: lower index).  idx_dev: k int32,    *
 * E_dev: k doubles.  1 <= k <= min(B, 1024).  E_approx_dev must hold no NaN *
 * (-0 and +0 are equal).  Up to 512 configurations the selection ranks      *
 * every pair; above, a radix select over an order-preserving 64-bit key of *
 * E (six 11-bit digit passes, then an ordered compaction) does it in O(B).  */
goac_status goac_topk_rescore(goac_problem* prob, const int8_t* species_dev, int32_t B, const double* E_approx_dev,
                              int32_t k, int32_t* idx_dev, double* E_dev);

/* Random valid structures (SI, Random (R)): each class receives its multiset *
 * of species in uniformly random order (Fisher-Yates; draw t of class k for  *
 * configuration b is word t%4 of Philox4x32-10(ctr={t/4, b, k, 5}, seed)).   */
goac_status goac_random_configs(goac_problem* prob, int32_t B, uint64_t seed, int8_t* species_dev);

/* ------------------------------------------------------------------------ *
 * Parallel-chain Metropolis swap Monte Carlo (SI, Monte Carlo): chain c,    *
 * step t draws x = Philox4x32-10(ctr = {t_lo, t_hi, c, 0}, key = seed);     *
 * class: the only movable class, else word 0 of Philox(ctr={t_lo,t_hi,c,1})  *
 * with weight n_k(n_k - 1); positions a = (x0 n)>>32, b' = (x1 (n-1))>>32,   *
 * b = b' + (b' >= a); u = ((x2>>5) 2^26 + (x3>>6)) 2^-53.  Equal species: a  *
 * no-op.  Accept iff dE <= 1e-9 eV or u < exp(-dE/kT) (kT <= 0: the first  *
 * test only; |dE| <= 1e-9 eV is read as dE = 0, the rounding of symmetric   *
 * swaps),                                                                   *
 *   dE = 2 d (phi_a - phi_b) + d^2 (J_aa + J_bb - 2 J_ab), d = q_b - q_a,    *
 * phi = J q held per chain; on acceptance phi += d (J_:a - J_:b).           *
 *   species_dev: C x Nv in/out.  kT_dev: C.  Steps step0 .. step0+n_steps-1 *
 *   (resuming at step0 continues the same stream).  E_dev, bestE_dev: C     *
 *   doubles out (best: the last energy that undercut every earlier one by   *
 *   more than the 1e-9 eV tie, so that which of several symmetry-equivalent *
 *   configurations is kept does not follow rounding); best_species_dev:     *
 *   C x Nv out (nullable), the configuration of that energy; n_accept_dev: C *
 *   int64 out (nullable).  precision: GOAC_PREC_F64 (trajectory-exact to    *
 *   the FP64 definition) or GOAC_PREC_F32 (phi and J rows in FP32).         *
 *   GOAC_ERR_INVALID_ARG when no class has two positions (no swap exists).   *
 * ------------------------------------------------------------------------ */
goac_status goac_mc_run(goac_problem* prob, int8_t* species_dev, int32_t C, const double* kT_dev, int64_t n_steps,
                        uint64_t seed, uint64_t step0, int32_t precision, double* E_dev, double* bestE_dev,
                        int8_t* best_species_dev, int64_t* n_accept_dev);

/* Run-level stop and statistics of the Monte Carlo chains (Section         *
 * "Internal Fortran Heuristics in GOAC": a run ends after a given number of *
 * steps, or of steps without improvement).  goac_mc_run with:               *
 *   patience: with patience > 0 a chain stops after step t once             *
 *     t - t_imp >= patience, t_imp being the last step whose acceptance      *
 *     lowered E by more than 1e-9 eV below E at the previous such step (the  *
 *     start, step0 - 1, counts as one); 0 = run all n_steps.                 *
 *   stats (nullable; each pointer nullable, device arrays of C int64):       *
 *     n_accept_dev accepted swaps; n_noop_dev proposals of two positions     *
 *     holding the same species; best_step_dev the step at which the chain    *
 *     first reached its best energy (step0 - 1: the starting configuration); *
 *     steps_dev the steps run (< n_steps when patience stopped the chain).   *
 * The other arguments are those of goac_mc_run.                              */
typedef struct goac_mc_stats {
    int64_t* n_accept_dev;
    int64_t* n_noop_dev;
    int64_t* best_step_dev;
    int64_t* steps_dev;
} goac_mc_stats;
goac_status goac_mc_run_ex(goac_problem* prob, int8_t* species_dev, int32_t C, const double* kT_dev, int64_t n_steps,
                           uint64_t seed, uint64_t step0, int32_t precision, int64_t patience, double* E_dev,
                           double* bestE_dev, int8_t* best_species_dev, const goac_mc_stats* stats);

/* Launch-shape autotuner for goac_mc_run / goac_sa_run / goac_remc_run (no *
 * counterpart in the paper): each (warps per chain W, chains per CTA) in     *
 * {1, 2, 4} x {1, 2, 4, 8, 15} that fits in shared memory runs probe_steps  *
 * steps on a scratch copy of species_dev (C x Nv, not modified) with the    *
 * temperatures kT_dev (C); the fastest (CUDA events on the context stream)  *
 * is kept in the problem for `precision` and used by later calls.  The      *
 * trajectories do not depend on the launch shape.  W_out, cpc_out, ms_out   *
 * (host, nullable): the choice and its probe time.  Synchronises.           */
goac_status goac_mc_autotune(goac_problem* prob, const int8_t* species_dev, int32_t C, const double* kT_dev,
                             int64_t probe_steps, int32_t precision, int32_t* W_out, int32_t* cpc_out,
                             double* ms_out);

/* Set the launch shape that goac_mc_autotune would choose (no counterpart  *
 * in the paper): W warps per chain (1, 2 or 4) and chains_per_cta (1..32,   *
 * capped by shared memory and 1,024 threads) for `precision` (F64 or F32);  *
 * 0 restores the size-based choice for that field.  Host only; later         *
 * goac_mc_run / goac_sa_run / goac_remc_run calls of the problem use it.    *
 * The trajectories do not depend on the launch shape.                        */
goac_status goac_mc_set_shape(goac_problem* prob, int32_t precision, int32_t W, int32_t chains_per_cta);

/* Simulated annealing (SI, Simulated annealing: the MC routine with the     *
 * temperature lowered towards 0 during the run): goac_mc_run with the        *
 * temperature of step t set to kT0 (kT1/kT0)^(t/(total_steps-1)) per chain   *
 * (an exponential schedule, as in the paper's runs).  kT0_dev, kT1_dev: C.   */
goac_status goac_sa_run(goac_problem* prob, int8_t* species_dev, int32_t C, const double* kT0_dev,
                        const double* kT1_dev, int64_t total_steps, int64_t n_steps, uint64_t seed, uint64_t step0,
                        int32_t precision, double* E_dev, double* bestE_dev, int8_t* best_species_dev,
                        int64_t* n_accept_dev);

/* Gradient descent over single-swap neighbours (SI, Gradient Descent), for a *
 * batch of B configurations (species_dev B x Nv, in/out).  Each step          *
 * evaluates dE for every pair a < b of the same class holding different      *
 * species; if the minimum dmin < -1e-9 eV, the lowest pair (a, b)            *
 * (lexicographic) with dE <= dmin + 1e-9 eV is swapped, else the             *
 * configuration is a local minimum and stays.  At most max_steps steps.       *
 * E_dev: B final energies (FP64); steps_dev: B int64 steps taken.            *
 * Synchronises every 8 steps to stop once every configuration has converged. */
goac_status goac_gd_run(goac_problem* prob, int8_t* species_dev, int32_t B, int32_t max_steps, double* E_dev,
                        int64_t* steps_dev);

/* Replica-exchange Monte Carlo (SI, Replica Exchange Monte Carlo): G groups  *
 * of R chains (chain c = g R + slot; species_dev is G R x Nv, in/out).  Each *
 * round runs steps_per_round Metropolis steps per chain at its current       *
 * temperature (steps r*steps_per_round ...), then neighbouring temperature   *
 * ranks (k, k+1), k = r%2, r%2 + 2, ..., exchange with probability           *
 * min[1, exp(dE (1/kT_k - 1/kT_{k+1}))], dE = E(rank k) - E(rank k+1), u from *
 * words 0,1 of Philox(ctr = {r, g, k, 6}); an exchange swaps the two chains' *
 * temperatures.  kT_ladder_host: R temperatures (> 0).  E_dev: G R energies;  *
 * perm_dev: G R int32, chain holding rank k of group g at [g R + k];          *
 * n_exchanges_host: accepted exchanges (nullable; synchronises if given).     */
goac_status goac_remc_run(goac_problem* prob, int8_t* species_dev, int32_t G, int32_t R, const double* kT_ladder_host,
                          int32_t n_rounds, int64_t steps_per_round, uint64_t seed, int32_t precision, double* E_dev,
                          int32_t* perm_dev, int64_t* n_exchanges_host);

/* Hybrid heuristic (SI, Hybrid Methods: REMC and GA called alternately, the  *
 * best solutions passed on): n_cycles of goac_remc_run on the P = G R        *
 * configurations (key seed + 2c), each followed by n_gen GA generations with *
 * FP64 rescoring (goac_ga_run, key seed + 2c + 1, generations from c n_gen)  *
 * starting from the REMC configurations; the GA population (elites first)    *
 * starts the next cycle.  `precision` applies to the MC segments.  E_dev: P  *
 * final energies.  Synchronises.                                              */
goac_status goac_hybrid_run(goac_problem* prob, int8_t* species_dev, int32_t G, int32_t R,
                            const double* kT_ladder_host, int32_t n_cycles, int32_t n_rounds, int64_t steps_per_round,
                            int32_t n_gen, int32_t n_elite, uint32_t p_mut_u32, uint64_t seed, int32_t precision,
                            double* E_dev);

/* ------------------------------------------------------------------------ *
 * Batched Monte Carlo over many independent problems in one persistent      *
 * launch (the paper runs independent heuristic runs in parallel, Section    *
 * "Internal Fortran Heuristics in GOAC").  For problem p: chains[p] chains, *
 * species_dev[p] (chains[p] x Nv_p, in/out), kT_dev[p] (chains[p]),         *
 * E_dev[p] / bestE_dev[p] (chains[p], out), seed + p as the Philox key.     *
 * Host arrays of length n_probs hold the per-problem pointers.  Each chain  *
 * is the same stream as goac_mc_run with that problem and key.  A device    *
 * work queue hands (problem, chain) items to warps; no spin-waits.          *
 * use_graph != 0 captures the launch sequence in a CUDA graph (replayed on  *
 * later calls with the same arguments).                                      *
 * ------------------------------------------------------------------------ */
goac_status goac_batch_mc_run(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs,
                              int8_t* const* species_dev, const int32_t* chains, const double* const* kT_dev,
                              int64_t n_steps, uint64_t seed, uint64_t step0, int32_t precision,
                              double* const* E_dev, double* const* bestE_dev, int32_t chains_per_cta,
                              int32_t mode);

/* Autotuner for goac_batch_mc_run (the batching form's chains-per-CTA): runs *
 * each candidate 1, 2, 4, 8, 16, 32 that fits in shared memory for          *
 * probe_steps steps on scratch copies of the chains (the caller's            *
 * configurations are unchanged) in one persistent launch, times each with    *
 * CUDA events, and returns the fastest in best_chains_per_cta (and its time   *
 * in best_ms, nullable).  Synchronises.                                       */
goac_status goac_batch_mc_autotune(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs,
                                   int8_t* const* species_dev, const int32_t* chains, const double* const* kT_dev,
                                   int64_t probe_steps, int32_t precision, int32_t* best_chains_per_cta,
                                   double* best_ms);

/* ------------------------------------------------------------------------ *
 * Genetic algorithm, one generation (SI, Genetic Algorithm; roulette wheel *
 * selection).  pop_dev P x Nv with energies E_dev (P).  Children 0..e-1 are *
 * the n_elite lowest (E, index).  Roulette on F_b = floor((Emax - E_b) /     *
 * (Emax - Emin) 2^24) (all 1 if Emax == Emin): a 64-bit draw x picks the    *
 * first b whose running sum of F exceeds (x F_total) >> 64; parents of child *
 * c in generation gen: x_A = w0:w1, x_B = w2:w3 of Philox(ctr={0,gen,c,2}). *
 * Crossover from A: for each site i ascending with child_i != B_i, j = the  *
 * lowest site of i's class with child_j == B_i and B_j != B_i; candidate k  *
 * is taken iff word k%4 of Philox(ctr={k/4,gen,c,3}) < 2^31.  Mutation: if  *
 * w0 of Philox(ctr={0,gen,c,4}) < p_mut_u32, one swap (class from w1,       *
 * positions from w2, w3 as in the Monte Carlo pick).                         *
 *   children_dev P x Nv out; parents_dev (P x 2 int32) and nswap_dev        *
 *   (P x 2 int32: swaps taken, candidates) are optional outputs.  A child's  *
 *   working set lives in shared memory: Nv <= 33,432 (fewer with many        *
 *   species), else GOAC_ERR_INVALID_ARG.                                     *
 * ------------------------------------------------------------------------ */
goac_status goac_ga_generation(goac_problem* prob, const int8_t* pop_dev, const double* E_dev, int32_t P,
                               int32_t n_elite, uint32_t p_mut_u32, uint32_t gen, uint64_t seed,
                               int8_t* children_dev, int32_t* parents_dev, int32_t* nswap_dev);

/* GA run: scores pop_dev, then n_gen x (generation + rescoring of every     *
 * child with `precision`; with a tensor-core precision the FP64 energy is    *
 * used only through the split form).  pop_dev (P x Nv) and E_dev (P) are    *
 * in/out.  Generations are numbered gen0, gen0 + 1, ...                     *
 * GOAC_PREC_F64_INCR rescores incrementally in FP64 (the paper's GA keeps   *
 * the energies of its structures; the rescoring of a child from its parent *
 * is this library's reading): the potentials phi = J_vv q + phi_fix of the  *
 * population are formed once, and each child c takes the parent P (of its   *
 * two; ties: the first) from which it differs in fewer sites, then          *
 *   phi_c = phi_P + sum_{s: c_s != P_s} (z[c_s] - z[P_s]) J_vv[s][:]        *
 * over the changed sites in ascending order and                             *
 *   E_c = sum_v q_c,v (phi_c,v + phi_fix,v) + E_const,                      *
 * equal to the full q^T J q to FP64 rounding.  Needs Nv <= 17066, else      *
 * GOAC_ERR_UNSUPPORTED.                                                     */
goac_status goac_ga_run(goac_problem* prob, int8_t* pop_dev, double* E_dev, int32_t P, int32_t n_gen,
                        int32_t n_elite, uint32_t p_mut_u32, uint64_t seed, uint32_t gen0, int32_t precision);

/* GA run with the run-level stops of Section "Internal Fortran Heuristics in *
 * GOAC" (a run ends after a number of generations, or of generations        *
 * without improvement, or a time budget) and the n lowest structures as      *
 * output (Section "Implementation and Theoretical Background").  R           *
 * populations of params->P in pop_dev (R P x Nv) and E_dev (R P), each       *
 * evolving as goac_ga_run with key seed + r (goac_ga_run_populations).       *
 * Patience: after generation g the population's lowest energy b_g improves  *
 * when b_g < b_ref - 1e-9 eV, b_ref the lowest energy at the previous       *
 * improvement (at first the initial population's); with patience > 0 a      *
 * population stops once `patience` generations in a row brought none (later *
 * generations leave it unchanged).  time_budget_s > 0: the host checks the   *
 * wall clock every 8 generations and stops there once it is spent.          *
 * topk > 0 (<= min(P, 1024)): the topk lowest of each final population,      *
 * rescored in FP64 and sorted (goac_topk_rescore), into top_idx_dev (R topk  *
 * int32, indices within the population) and topE_dev (R topk doubles).       *
 * stats_host (nullable): R entries.  Synchronises when patience, a time      *
 * budget or stats are given.                                                 */
typedef struct goac_ga_params {
    int32_t P;               /* individuals per population                      */
    int32_t n_gen;           /* most generations                                */
    int32_t n_elite;         /* the n_elite lowest (E, index) survive            */
    uint32_t p_mut_u32;      /* mutation probability x 2^32                      */
    int32_t precision;       /* rescoring form, GOAC_PREC_* (F64_INCR included) */
    int32_t patience;        /* generations without improvement (0: no limit)   */
    uint32_t gen0;           /* number of the first generation (draw counter)   */
    double time_budget_s;    /* host wall-clock budget in seconds (0: none)     */
} goac_ga_params;
typedef struct goac_ga_stats {
    int32_t generations;     /* generations run                                 */
    int32_t best_generation; /* generation of the last improvement (0: none)    */
    int32_t stop_reason;     /* 0: n_gen reached, 1: patience, 2: time budget    */
    int32_t reserved;
    double best_E;           /* lowest energy of the final population            */
} goac_ga_stats;
goac_status goac_ga_run_ex(goac_problem* prob, int8_t* pop_dev, double* E_dev, int32_t R,
                           const goac_ga_params* params, uint64_t seed, int32_t topk, int32_t* top_idx_dev,
                           double* topE_dev, goac_ga_stats* stats_host);

/* R independent GA populations of P configurations each (the paper compares  *
 * independent runs of its heuristics; this runs them together): population  *
 * r occupies rows r P .. r P + P - 1 of pop_dev (R P x Nv) and E_dev (R P)   *
 * and evolves exactly as goac_ga_run with key seed + r would on it alone     *
 * (selection, elitism, crossover and mutation within the population; parent *
 * indices population-local).  Every generation's children of all            *
 * populations come from one launch and are rescored by one call over R P     *
 * configurations.  R P <= GOAC_MAX_BATCH.                                    */
goac_status goac_ga_run_populations(goac_problem* prob, int8_t* pop_dev, double* E_dev, int32_t R, int32_t P,
                                    int32_t n_gen, int32_t n_elite, uint32_t p_mut_u32, uint64_t seed, uint32_t gen0,
                                    int32_t precision);

/* GA populations of several problems of different sizes in one launch per   *
 * step (the batching form; the paper compares independent runs of its        *
 * heuristics): problem i evolves the population pop_dev[i] (P[i] x Nv_i,     *
 * in/out) with energies E_dev[i] (P[i], out) exactly as goac_ga_run with key *
 * seed + i and the common n_gen, n_elite (<= every P[i]), p_mut_u32, gen0.   *
 * Each generation's select, elite, children and rescoring kernels serve all  *
 * populations at once.  precision: GOAC_PREC_F64_INCR (incremental FP64      *
 * rescoring) only.  Every problem belongs to ctx and appears once; host      *
 * arrays of length n_probs.                                                  */
goac_status goac_batch_ga_run(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs, int8_t* const* pop_dev,
                              double* const* E_dev, const int32_t* P, int32_t n_gen, int32_t n_elite,
                              uint32_t p_mut_u32, uint64_t seed, uint32_t gen0, int32_t precision);

/* ------------------------------------------------------------------------ *
 * Relaxed occupations (differentiable form; the paper's descent is discrete,*
 * SI Gradient Descent).  logits_dev: B x Nv x S float; p = softmax over the *
 * species allowed in each site's class; q_v = sum_s p_vs z_s;               *
 *   E = q^T J q + lambda sum_{k,s allowed} (sum_{v in k} p_vs - n_ks)^2,    *
 *   g_vs = z_s (2 J q)_v + 2 lambda (sum_{w in k} p_ws - n_ks),             *
 *   dE/dL_vs = p_vs (g_vs - sum_t p_vt g_vt)  (0 for masked species).       *
 * E_dev: B doubles; dlogits_dev: B x Nv x S floats (nullable).  precision: *
 * GOAC_PREC_F64 (FP64 CUDA-core GEMM), GOAC_PREC_TF32X2 (J.Q on tcgen05,  *
 * J and the real-valued Q each split in TF32 hi / lo, the products hi.hi,   *
 * hi.lo and lo.hi accumulated in FP32; Phi kept in FP32) or                 *
 * GOAC_PREC_F16X2 (the same three products with FP16 hi / lo parts, J      *
 * scaled per 128-row panel by a power of two into FP16's range: the same   *
 * 11-bit parts as TF32, at the FP16 tensor rate, twice TF32's).            *
 * ------------------------------------------------------------------------ */
goac_status goac_energy_grad(goac_problem* prob, const float* logits_dev, int32_t B, double lambda,
                             int32_t precision, double* E_dev, float* dlogits_dev);

/* Projected descent on the logits (the relaxed, differentiable form; the    *
 * paper's own gradient descent is discrete, SI Gradient Descent; used to     *
 * seed MC / GA populations): n_steps of L -= eta dE/dL with the gradient of  *
 * goac_energy_grad (softmax keeps p on the simplex), in place on logits_dev. *
 * precision: as goac_energy_grad; with TF32X2 and F16X2 the chain-rule       *
 * kernel applies each step itself.  dlogits_scratch_dev: caller buffer of    *
 * B x Nv x S floats, not NULL (the F64 path's gradient).  E_dev: energies    *
 * after the last step.                                                       */
goac_status goac_relaxed_descent(goac_problem* prob, float* logits_dev, int32_t B, double lambda, double eta,
                                 int32_t n_steps, int32_t precision, float* dlogits_scratch_dev, double* E_dev);

/* Relaxed occupations p = softmax of the logits over the species allowed in  *
 * each site's class (FP64 inside, FP32 out): logits_dev, p_dev B x Nv x S.   */
goac_status goac_occupations(goac_problem* prob, const float* logits_dev, int32_t B, float* p_dev);

/* Round relaxed occupations p (B x Nv x S float) to valid configurations:    *
 * per class, (site, species) pairs by p descending (ties: lower site, then   *
 * lower species) are assigned when the site is free and the species quota   *
 * is left.  species_dev: B x Nv int8 out.                                    */
goac_status goac_round_to_counts(goac_problem* prob, const float* p_dev, int32_t B, int8_t* species_dev);

#ifdef __cplusplus
}
#endif
#endif /* GOAC_H */
