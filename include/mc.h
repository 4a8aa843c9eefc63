/*
 * mc.h -- C ABI of the GB300 sequential-Metropolis library (libmcgb300.so).
 *
 * The library runs the canonical Metropolis Monte Carlo of primitive-model
 * electrolytes of Liang, Xing & Li (arXiv:1602.05716): ions are hard spheres
 * of diameter sigma carrying integer valences q, interacting by the bare
 * Coulomb potential l_B q_i q_j / r in units of k_B T (l_B = Bjerrum length),
 * no cutoff and no periodic images, confined by a hard spherical wall of
 * radius R (Sec. 5.2).  One sweep ("Monte Carlo cycle") tries every ion once
 * in ascending index order (Sec. 2, sequential updating scheme); each trial
 * move draws a displacement uniform in a cube of half-width h (Algorithm 1),
 * computes the exact O(N) energy change
 *     dE = l_B q_i sum_{j != i} q_j (1/|x'_i - x_j| - 1/|x_i - x_j|)
 * against the current positions of all other ions (Sec. 2, the Delta E_ij
 * table), rejects on hard-core overlap (Sec. 3.3) or the wall, and accepts
 * when the uniform draw u satisfies u < exp(-dE) (Algorithm 4, Eq.
 * trial-outcome).
 *
 * Decisions and positions are bit-identical to the FP64 CPU oracle that uses
 * the same Philox4x32-10 stream keyed by (seed, chain) with counter = move
 * index; the GPU computes pair terms in FP32 and recomputes a move's dE in the
 * oracle's FP64 arithmetic whenever the FP32 value lies inside its proven
 * error bound of the acceptance threshold.
 *
 * Conventions for every call:
 *  - Return 0 (MC_OK) on success, a negative MC_ERR_* code otherwise; the
 *    message of the last failure on the calling thread is mc_last_error().
 *  - Host pointers are read (or written) only during the call; the caller
 *    keeps ownership.  Positions are float32, packed xyz (3 floats per ion),
 *    ion-major; valences are float32 (integer values).
 *  - A handle owns its device memory and a CUDA stream; calls on one handle
 *    must not run concurrently from several host threads.
 *  - After MC_ERR_TIMEOUT or MC_ERR_CUDA from a sweep the handle is poisoned
 *    (every later call but mc_destroy/mc_last_error returns MC_ERR_POISONED);
 *    the device itself stays usable for other handles.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_ERR_INVALID (-1)      /* bad argument (NULL pointer, N < 1, sigma <= 0, ...) */
#define MC_ERR_OVERLAP_INIT (-2) /* input configuration overlaps or leaves the wall */
#define MC_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define MC_ERR_TIMEOUT (-4)      /* a bounded device-side wait expired */
#define MC_ERR_OOM (-5)          /* device or host allocation failed */
#define MC_ERR_POISONED (-6)     /* handle unusable after an earlier TIMEOUT/CUDA error */

typedef struct mc_system *mc_handle;

/* One chain's inputs (mc_create_batch).  pos_xyz: n*3 floats; q: n floats. */
typedef struct {
    const float *pos_xyz;
    const float *q;
    int64_t n;
    double sigma;      /* hard-core diameter */
    double l_B;        /* Bjerrum length, in units of length (same as sigma) */
    double R;          /* radius of the hard spherical wall; centres stay within R - sigma/2 */
    double half_width; /* h: trial displacement uniform in [-h, h)^3 */
    uint64_t seed;     /* Philox key (low 32 bits) and counter word 3 (high 32 bits) */
    uint32_t chain_id; /* Philox key word 1 */
} mc_chain_desc;

/* Counters of one chain since creation (mc_stats). */
typedef struct {
    uint64_t sweeps;         /* completed sweeps */
    uint64_t accepts;        /* accepted moves */
    uint64_t rej_metropolis; /* rejected by u >= exp(-dE) */
    uint64_t rej_overlap;    /* rejected by hard-core overlap */
    uint64_t rej_wall;       /* rejected by the wall */
    uint64_t guard_fp64;     /* moves sent to the guard tiers (FP32 value inside its error band) */
    uint64_t decided_interval; /* moves decided before the outcomes of earlier moves of their group were known */
    uint64_t tier2, tier3, tier4; /* guard decisions by accurate FP32, double-single, FP64 */
    uint64_t rounds;         /* decision rounds over all work items */
    uint64_t cyc_wait_window; /* SM cycles, summed over work items: waiting for the previous group's outcome, */
    uint64_t cyc_tiles;      /* ... in the pair-sum tiles (including waits for their publication), */
    uint64_t cyc_resolve;    /* ... deciding (rounds, excluding guard tiers), */
    uint64_t cyc_guard;      /* ... in guard tiers, */
    uint64_t cyc_total;      /* ... and in total */
    uint64_t cyc_tier[3];    /* SM cycles in guard tiers 2, 3 and 4 */
    uint64_t ovl_scan;       /* exact overlap scans (FP32 minimum inside the overlap band) */
    uint64_t cyc_ovl_scan;   /* SM cycles in those scans */
    uint64_t da_rej1;        /* delayed acceptance: moves rejected by the surrogate stage */
    uint64_t da_ovl1;        /* ... overlaps found by the surrogate stage (counted in rej_overlap too) */
    uint64_t da_fp64;        /* ... surrogate energy changes recomputed in the reference FP64 arithmetic */
    uint64_t cyc_da1;        /* ... SM cycles in the surrogate stage, summed over work items, */
    uint64_t cyc_da_part[4]; /* ... of which: [2] the MLP, [3] the near field with its shell histograms
                                ([0] and [1] stay 0) */
    uint64_t drift_checks;   /* periodic drift checks run (MC_OPT_DRIFT_EVERY) */
    double drift_last;       /* |ledger - E| at the last check, E the accurate recomputed energy */
    double drift_max;        /* largest |ledger - E| over the checks */
} mc_stats_t;

/* Per-move validation record (mc_record_enable / mc_record_read). */
typedef struct {
    uint64_t m;     /* move index = sweep * N + i */
    int32_t i;      /* ion */
    int32_t outcome; /* 0 accept, 1 Metropolis reject, 2 overlap, 3 wall, 4 rejected by the surrogate stage */
    double dE;      /* dE used for the ledger / decision (FP64 value when tier == 4); NaN if not evaluated */
    double dE32;    /* dE from the FP32 pair sums (NaN when not evaluated) */
    double bound;   /* proven bound of |dE32 - dE_FP64| apart from a relative 2^-20 |dE| (the static band of
                       the FP32 decision); +inf when a guard mode disabled the band */
    double dEt;     /* delayed acceptance: the surrogate energy change (the reference FP64 value where it was
                       computed, else FP32); NaN for plain moves and moves the surrogate did not evaluate */
    int32_t tier;   /* 0 decided from an interval, 1 from the exact FP32 sum, 2 accurate FP32, 3 double-single,
                       4 the FP64 recomputation, 5 overlap found by the exact overlap scan; delayed acceptance:
                       6 decided by the surrogate stage in FP32, 7 ... in the reference FP64 arithmetic */
    int32_t pad;
} mc_record;

/* Create a single chain (a batch of one).  Copies pos_xyz (n*3) and q (n) to
 * the device, validates that every centre lies within R - sigma/2 and no two
 * centres are closer than sigma (MC_ERR_OVERLAP_INIT otherwise), and computes
 * the initial energy for the ledger.  Sec. 3.1 (float4 x,y,z,valence layout),
 * Sec. 5.2 (spherical hard wall).                                            */
int mc_create(const float *pos_xyz, const float *q, int64_t n, double sigma, double l_B, double R,
              double half_width, uint64_t seed, uint32_t chain_id, mc_handle *out);

/* Create n_chains independent chains (uneven N allowed) swept together by one
 * persistent launch.  Chains are addressed by index 0..n_chains-1 below.
 * The paper runs one independent simulation per GPU (Sec. 5.2); here many
 * independent chains share one GPU.                                          */
int mc_create_batch(const mc_chain_desc *descs, int n_chains, mc_handle *out);

/* Run n_sweeps sweeps of every chain of the handle (Sec. 2; Algorithms 1-5
 * describe the paper's GPU schedule, which this launch replaces by its own).
 * Blocks until done; returns MC_ERR_TIMEOUT if a device-side wait expired.  */
int mc_sweep(mc_handle h, int64_t n_sweeps);

/* Enqueue n_sweeps sweeps on the handle's stream and return; errors surface
 * at the next mc_synchronize.                                               */
int mc_sweep_async(mc_handle h, int64_t n_sweeps);
int mc_synchronize(mc_handle h);

/* Use the caller's CUDA stream (a cudaStream_t passed as void*); NULL reverts
 * to the handle's own stream.                                                */
int mc_set_stream(mc_handle h, void *cuda_stream);

/* Energy of chain `chain`: *ledger = initial energy + sum of accepted dE (FP64
 * running ledger); *recomputed (nullable) = l_B sum_{i<j} q_i q_j / r_ij of the
 * current configuration (the drift check), every term in float-float
 * arithmetic: exact coordinate differences, a float-float squared distance,
 * one Newton step on rsqrt (about 2e-14 relative per term), FP64 sums in a
 * fixed order that depends on N only.  The initial ledger is the same
 * computation.  Sec. 5.2 monitors the total energy to judge equilibration.  */
int mc_energy(mc_handle h, int chain, double *ledger, double *recomputed);

/* Pair-distance histogram behind g_{++}, g_{+-}, g_{--} (Sec. 5.2, Fig. PCF).
 * For every ion i with |r_i| <= R - sigma/2 - wall_margin (all ions when
 * wall_margin <= 0) and every j != i: bin = floor(r_ij / (r_max / n_bins)),
 * counted when bin < n_bins.  counts has 3*n_bins entries (class-major:
 * 0 = both valences > 0, 1 = mixed, 2 = both < 0) and is ADDED to (caller-
 * owned, accumulate over calls).  r_ij is the FP64 distance of the FP32
 * centres, so counts are exact integers.                                     */
int mc_gr_histogram(mc_handle h, int chain, int n_bins, double r_max, double wall_margin, uint64_t *counts);

/* Copy chain positions to / from a caller buffer of n*3 floats (pinned host
 * memory makes the copies direct).  Setting validates like mc_create
 * (MC_ERR_OVERLAP_INIT), with the same FP64 rule applied on the device (the
 * wall, and every pair closer than sigma found through a grid of cells of
 * edge >= sigma); on failure the chain keeps its positions.  The ledger is
 * kept as it is.  The first call allocates the chain's staging and grid
 * (12 n bytes, and up to 4 n cells of a few slots each).                    */
int mc_get_positions(mc_handle h, int chain, float *pos_xyz);
int mc_set_positions(mc_handle h, int chain, const float *pos_xyz);

/* Checkpoint: positions (n*3 floats), completed sweeps, energy ledger and
 * counters.  Restoring them (with the same seed/chain id) resumes the chain
 * bit-identically, because every random draw is keyed by the move index.    */
int mc_get_state(mc_handle h, int chain, float *pos_xyz, uint64_t *sweeps, double *ledger, mc_stats_t *stats);
int mc_set_state(mc_handle h, int chain, const float *pos_xyz, uint64_t sweeps, double ledger,
                 const mc_stats_t *stats);

/* Counters of chain `chain` (accepts, rejects by cause, FP64 guard count). */
int mc_stats(mc_handle h, int chain, mc_stats_t *out);

/* Number of chains and N of a chain. */
int mc_num_chains(mc_handle h);
int64_t mc_num_ions(mc_handle h, int chain);

/* Validation mode: record the first `cap` moves of later sweeps of chain
 * `chain` (record index = sweeps since enabling * N + i).  cap = 0 disables. */
int mc_record_enable(mc_handle h, int chain, int64_t cap);
/* Copy up to cap records; returns the number copied (>= 0) or an error. */
int64_t mc_record_read(mc_handle h, int chain, mc_record *out, int64_t cap);

/* Work-item timeline (profiling): for each (sweep, group of 128 ions) of
 * chain `chain` after enabling, %globaltimer nanoseconds at which the work
 * item started, had everything but the previous group's outcome, observed
 * that outcome, finished deciding, published its own outcome, and published
 * its new positions.                                                        */
typedef struct {
    uint64_t item; /* sweep * groups + group */
    uint64_t t_start, t_ready, t_window, t_resolved, t_published;
    uint64_t n_guard; /* 1 if a guard tier ran */
    uint64_t t_positions; /* ... and published its new positions */
    uint64_t t_tile;      /* observed the last other group's positions (0: already published at the start) */
    uint64_t t_tiles;     /* finished the pair sums over the other groups */
    uint64_t t_w2;        /* observed the outcome of the group two before (0: none) */
    uint64_t t_ph[4];     /* pair sums combined, bands ready, round 0 done, oldest deep window's outcome observed */
    uint32_t c_res[8];    /* SM cycles from the window's outcome to: window sums, exact window terms, first round,
                             last round, resolved, outcome published, positions published, rounds run */
} mc_trace_rec;
int mc_trace_enable(mc_handle h, int chain, int64_t cap);
int64_t mc_trace_read(mc_handle h, int chain, mc_trace_rec *out, int64_t cap);

/* Energy series (Sec. 5.2: the total energy E_k monitored step by step).
 * After enabling, the sweep kernel stores the FP64 ledger (the energy of the
 * initial configuration plus every accepted dE) once the last group of each
 * sweep has been folded into it: entry k is E after the (k+1)-th sweep from
 * enabling, for the first `cap` sweeps (cap = 0 disables; the buffer is
 * device memory owned by the library).  Read copies min(cap, enabled
 * capacity, sweeps run since enabling) entries into the caller's host
 * buffer and returns how many (>= 0) or an error.                           */
int mc_energy_series_enable(mc_handle h, int chain, int64_t cap);
int64_t mc_energy_series_read(mc_handle h, int chain, double *out, int64_t cap);

/* Energy autocorrelation and integrated autocorrelation time (Sec. 5.2's
 * definitions): with E-bar the mean over the ensemble and the steps,
 *   C_n = <(E_k - E-bar)(E_{k+n} - E-bar)> / <(E_k - E-bar)^2>,
 * the numerator averaged over every series and every k with k + n inside
 * the series, the denominator over every entry; T_c = 1/2 + sum_{k=1}^{max_lag}
 * C_k (the paper's infinite sum, cut at max_lag by the caller).  Host only,
 * no device and no handle.  series: n_series rows of n_steps FP64 values,
 * row r at series + r * stride (caller-owned, read only); C: max_lag + 1
 * outputs (C[0] = 1); Tc may be NULL.  MC_ERR_INVALID for NULL pointers,
 * n_series < 1, n_steps < 2, stride < n_steps, max_lag outside
 * [0, n_steps), a non-finite entry, or a series without variance.         */
int mc_energy_autocorr(const double *series, int64_t n_series, int64_t n_steps, int64_t stride, int64_t max_lag,
                       double *C, double *Tc);

/* Dressed-ion analysis of pair correlations (Sec. 5.2): renormalised inverse
 * Debye length, valences and dielectric constant from the far field of
 * g_{++}, g_{+-}, g_{--}.  Reduced units: lengths in sigma, energies in k_BT,
 * eps = 1 / (4 pi l_B).  Host only, no device and no handle.
 *   counts     3 x n_bins pair counts as mc_gr_histogram returns them (++,
 *              mixed, --), summed over any number of configurations
 *   n_ref_p/m  the interior reference ions of each sign behind those counts
 *              (summed over the same configurations)
 *   dens_p/m   number densities of the positive and negative ions
 *   q_p, q_m   bare valences (q_p > 0 > q_m)
 *   r_lo..r_hi the far-field window: bins whose centre (k + 1/2) dr lies in it
 * Steps: g_ab(bin) = counts / (N_ref,a n_b V_bin) (mixed: counts /
 * ((N_ref,+ n_- + N_ref,- n_+) V_bin)); U_ab = -ln g_ab; rho^q_+ = n_+ q_+
 * g_{++} + n_- q_- g_{+-}, rho^q_- = n_+ q_+ g_{+-} + n_- q_- g_{--};
 * ln|r rho^q_+-| fitted by least squares with one common slope -kappa_R (and
 * each line's own slope); q^R from -kappa_R^2 U / (4 pi l_B rho^q) averaged
 * over the window, two ways for each sign; eps_R / eps from -kappa_R^2 q^R
 * e^{-kappa_R r} / (4 pi r rho^q) averaged likewise; and both sides of
 * (kappa_R / kappa)^2 = (q_+^R - q_-^R) / (q_+ - q_-).  Window bins with an
 * empty class or rho^q of the wrong sign (not screening) are skipped.
 *   g          (nullable) 3 x n_bins: the normalised g_ab (NaN where the
 *              normalisation is zero)
 *   out        the parameters; MC_ERR_INVALID for NULL counts/out, bad sizes
 *              or parameters, or fewer than 2 usable window bins.          */
typedef struct {
    double kappa;         /* bare: sqrt(4 pi l_B (n_+ q_+^2 + n_- q_-^2)) */
    double kappa_R;       /* common far-field slope of ln|r rho^q_+| and ln|r rho^q_-| */
    double kappa_R_pm[2]; /* each line's own slope: around a positive, around a negative ion */
    double qR_p[2];       /* q_+^R from U_{++} / rho^q_+ and from U_{-+} / rho^q_- */
    double qR_m[2];       /* q_-^R from U_{+-} / rho^q_+ and from U_{--} / rho^q_- */
    double epsR_pm[2];    /* eps_R / eps around a positive and a negative ion */
    double rd_lhs;        /* (kappa_R / kappa)^2 */
    double rd_rhs;        /* (q_+^R - q_-^R) / (q_+ - q_-), each q^R the mean of its two estimates */
    int64_t n_fit;        /* window bins used */
} mc_dit_result;
int mc_dressed_ion_analysis(const uint64_t *counts, int n_bins, double r_max, double n_ref_p, double n_ref_m,
                            double dens_p, double dens_m, double q_p, double q_m, double l_B, double r_lo,
                            double r_hi, double *g, mc_dit_result *out);

/* The parallel-reduction comparison code of Sec. 4, as a foil for mc_sweep:
 * one kernel launch per trial move, the N - 1 pair terms spread over blocks
 * of 1,024 threads (one pair each), block subtotals left in global memory and
 * counted by an atomic, the last block to finish deciding the move and
 * updating the ion.  With MC_SCHEME_SEQUENTIAL it runs the same exact chain
 * as mc_sweep (Sec. 2's sequential updating, the same draws and decisions
 * from sweep 0 of the description's positions), so after n sweeps its
 * positions equal those of mc_create + mc_sweep(n).  With MC_SCHEME_RANDOM it
 * runs Sec. 2's random updating scheme: cycle s has N steps, step t has move
 * index m = s N + t and moves ion floor(u N / 2^64), u = w1 2^32 + w0 from
 * the Philox draws of purpose 3 at m (trial and acceptance draws as in the
 * sequential scheme, purpose 0 at m).  Each cycle's N launches replay from
 * one CUDA graph for N <= 65,536 (plain launches above).  Blocks until done.
 *   desc      one chain, validated as by mc_create (caller-owned, read only)
 *   scheme    MC_SCHEME_SEQUENTIAL or MC_SCHEME_RANDOM
 *   pos_out   N x 3 floats, host, caller-owned: the positions after the sweeps
 *   dE_sum    (nullable) FP64 sum of the accepted moves' dE
 *   counts    (nullable) 5 counters: accepted, rejected by the Metropolis
 *             test, by overlap, by the wall, and moves whose tree sum fell
 *             within its rounding bound of the threshold and were re-summed
 *             in the canonical order
 *   ms        (nullable) CUDA-event time of the sweeps on the call's stream
 * Device memory is allocated and released inside the call.  Errors as
 * mc_create, MC_ERR_INVALID for n_sweeps < 0, an unknown scheme or a NULL
 * pos_out.                                                                   */
#define MC_SCHEME_SEQUENTIAL 0
#define MC_SCHEME_RANDOM 1
int mc_reduction_run(const mc_chain_desc *desc, int64_t n_sweeps, int scheme, float *pos_out, double *dE_sum,
                     uint64_t *counts, double *ms);

/* Options (mc_set_option):
 *  MC_OPT_GUARD_MODE   0 = FP32 with proven error band (default),
 *                      1 = recompute every evaluated move in FP64,
 *                      2 = decide from FP32 alone (band 0; test of the band only),
 *                      3 = send every evaluated move through the guard tiers
 *                          (accurate FP32, then double-single, then FP64)
 *  MC_OPT_TIMEOUT_MS   bound of every device-side wait (default 4000)
 *  MC_OPT_CTAS         persistent CTAs per launch (0 = one per resident slot)
 *  MC_OPT_SKIP_PUBLISH fault injection: the work item with this index never
 *                      publishes its result (waiters time out); -1 = off
 *  MC_OPT_USE_GRAPH    1 = capture each distinct sweep count in a CUDA graph
 *                      and replay it (default 1), 0 = plain launches
 *  MC_OPT_POLICY       order of the work items of a batch: 0 = one group of
 *                      every chain in turn (default), 1 = sweep-synchronous
 *  MC_OPT_DA           1 = chains with a surrogate (mc_set_surrogate) sweep with
 *                      delayed acceptance (default), 0 = they sweep plainly (the
 *                      surrogate stays set for mc_da_samples)
 *  MC_OPT_PAIRS        -1 = automatic (default: on for a single chain without a
 *                      surrogate of at most 2 x SMs groups when deep windows are
 *                      on), 0 = off, 1 = on:
 *                      thread-block clusters of two CTAs share each work item,
 *                      the second summing every other tile for the first.  The
 *                      trajectory is identical either way; reading it returns
 *                      whether the mode is in effect.
 *  MC_OPT_DEEP_WINDOWS 1 = on (default), 0 = off: the three groups before the
 *                      window are also computed for both positions, their
 *                      corrections held in tensor memory, so a group waits for
 *                      no tile later than five groups back.  The trajectory is
 *                      identical either way.
 *  MC_OPT_DRIFT_EVERY  K >= 1: inside each mc_sweep / mc_sweep_async call,
 *                      after every K completed sweeps, recompute every
 *                      chain's energy on the device (as mc_energy's
 *                      recomputed value) and store |ledger - E| in the
 *                      chain's drift_last, drift_max and drift_checks
 *                      (mc_stats); a call of fewer than K sweeps runs no
 *                      check.  Captured in the same CUDA graph as the sweeps.
 *                      0 = off (default).  The trajectory is unchanged.
 *  MC_OPT_HELPERS      0 = off (default), 1 = on when pairs mode is off:
 *                      launch the 512-thread form of the sweep kernel, whose
 *                      second 256 threads run half of every work item's pair
 *                      sums over the other groups with a small register
 *                      budget, while the first 256 run the work items as
 *                      before.  The trajectory is identical either way;
 *                      reading it returns whether the form is in effect.
 *                      The autotuner tries it.
 *  MC_OPT_DA_SWEEPS    sweeps per launch of chains with a surrogate or the
 *                      overlap prefilter (1 by default, at most 64): the cell
 *                      list is rebuilt at the start of each launch, so its
 *                      cells are sized for this many moves of every ion.
 *                      Set it before mc_set_surrogate / mc_set_overlap_prefilter
 *                      (MC_ERR_INVALID while a chain holds a cell list built
 *                      for another value).  The trajectory is unchanged.
 *  MC_OPT_SHARED_GUARD 1 = on (default), 0 = off.  In launches of chains
 *                      with a surrogate or the overlap prefilter, a move
 *                      whose FP32 value falls inside its error band is
 *                      recomputed (guard tiers 2 and 3) by its work item's
 *                      warps together with every warp of the launch that
 *                      waits at that moment, in chunks of 4096 partners,
 *                      instead of by its work item's CTA alone; one such
 *                      move at a time (others run on their own CTA).
 *                      Launches of plain chains only keep the tiers on the
 *                      work item's CTA.  Decisions and the trajectory are
 *                      unchanged; the dE recorded for a tier-2 or tier-3
 *                      move may differ in its last FP64 bits. */
#define MC_OPT_GUARD_MODE 1
#define MC_OPT_TIMEOUT_MS 2
#define MC_OPT_CTAS 3
#define MC_OPT_SKIP_PUBLISH 4
#define MC_OPT_USE_GRAPH 5
#define MC_OPT_POLICY 6
#define MC_OPT_DA 7
#define MC_OPT_PAIRS 8
#define MC_OPT_DEEP_WINDOWS 9
#define MC_OPT_DRIFT_EVERY 10
#define MC_OPT_HELPERS 11
#define MC_OPT_DA_SWEEPS 12
#define MC_OPT_SHARED_GUARD 13
int mc_set_option(mc_handle h, int option, int64_t value);
int mc_get_option(mc_handle h, int option, int64_t *value);

/* Autotuner: times trial_sweeps sweeps of every candidate and keeps the
 * fastest in the handle, restoring every chain's state, so the trajectories
 * are unchanged.  First the kernel shape at the current work order and CTA
 * count: pairs mode (MC_OPT_PAIRS), deep windows (MC_OPT_DEEP_WINDOWS) and
 * helper warps (MC_OPT_HELPERS), every combination the device and the chains
 * allow (pairs mode and helper warps exclude each other; pairs mode needs
 * clusters and no surrogate); then, with that shape, every work order
 * (MC_OPT_POLICY) and persistent CTA count (all resident slots, 3/4, 1/2).
 * Outputs (nullable): the chosen policy, CTA count, shape (bit 0 pairs
 * mode, bit 1 deep windows, bit 2 helper warps; the options are set to it)
 * and the winner's trial time in ms.  The paper tunes block size and
 * threads per particle by hand (Sec. 4, Table Para).                        */
int mc_autotune(mc_handle h, int64_t trial_sweeps, int64_t *best_policy, int64_t *best_ctas, int64_t *best_shape,
                double *best_ms);

/* ---- Delayed acceptance with a learned surrogate ----------------------
 * A two-stage Metropolis test (Christen & Fox, 2005) on the sequential chain of
 * Sec. 2 (the paper's method is the plain chain; this is an exact variant that
 * skips the O(N) sum of Eq. DeltaE for moves a cheap first stage rejects).
 * Counted ions of the move of ion i in group g = i / 128: every ion except i,
 * the earlier ions of g and the ions of the W groups tried just before g
 * (cyclic over the sweep); the set depends only on the move index.
 * Stage 1: a trial that overlaps a counted ion is rejected; otherwise the
 * surrogate energy change
 *     dEt = l_B q_i ([phi_near + g(v)](x') - [phi_near + g(v)](x))
 * decides: pass iff u1 == 0 or dEt < -ln u1 (u1 the plain chain's acceptance
 * draw, Philox purpose 0).  With d = |p - x_j| the FP64 distance of the FP32
 * centres, r_s = r_c / 2 and t = (d - r_s) / (r_c - r_s):
 *     phi_near(p) = sum over counted j with d^2 < r_c^2 of q_j s(d) / d,
 *     s(d) = 1 for d <= r_s, 1 - t^2 (3 - 2t) beyond (a C1 taper to 0 at r_c),
 * added in ascending j.  g is a 33-64-64-1 MLP, SiLU after both hidden layers,
 * BF16 weights, fed with
 *     v[k] = F_k / 4 (k < 32),  v[32] = |p| / R,
 * F_k the net valence of the counted ions in the taper region
 * r_s^2 <= d^2 < r_c^2 whose shell index floor(32 (d^2 - r_s^2) / (r_c^2 -
 * r_s^2)) (FP64, clamped to 31) is k: 32 shells of equal width in d^2.
 * Stage 2 (survivors only): the exact sum of the plain chain (overlap with any
 * ion rejects); accept iff u2 == 0 or dE - dEt < -ln u2, u2 the fourth word of
 * Philox purpose 1.  Decisions are those of the FP64 reference arithmetic, bit
 * for bit (FP32 with proven bands, the reference recomputation inside them).
 *
 * mc_set_surrogate installs the 6401 BF16 weights (layout W1[64][33], b1[64],
 * W2[64][64], b2[64], W3[64], b3; copied), the cutoff r_c (0 < r_c <= 5 sigma)
 * and W >= 2; the launch then uses at most W - 1 persistent CTAs.  w_bf16 =
 * NULL removes the surrogate.  Sweeps with a surrogate run one sweep per
 * launch after a preparation pass that builds a near-field cell list of the
 * sweep's start positions (no charge grid).                                  */
int mc_set_surrogate(mc_handle h, int chain, const uint16_t *w_bf16, int64_t n_w, double r_c, int W);

/* Overlap prefilter (an exact speed-up of the plain chain; Sec. 2's rule that a
 * trial overlapping another ion is rejected whatever its energy change).
 * Before any pair sum, each work item rejects the moves whose trial position
 * overlaps an ion it can already place: an ion more than W groups back in the
 * sweep, or a later ion of its own group.  They are found through a cell list
 * of the sweep's start positions (cells of edge at least (sigma + 2 sqrt(3)
 * h) / 2, every listed position kept current as moves are accepted; a cell
 * holds at most 64 ions and any beyond are simply not listed).  The plain
 * chain rejects those moves as overlaps too, so decisions, positions and
 * ledger are the plain chain's bit for bit; the surviving moves pay the O(N)
 * sum and are decided by the plain rule (draw purpose 0, the same band and
 * guard tiers).  Records of prefilter rejections carry tier 6.
 * W >= 2 sets it (the launch then uses at most W - 1 persistent CTAs, as with
 * a surrogate), W = 0 removes it.  Like a surrogate it makes sweeps run one
 * per launch after the cell list is rebuilt, MC_OPT_DA = 0 suspends it, and
 * it replaces a surrogate set on the chain (mc_set_surrogate replaces it in
 * turn).  Device memory: at most 8 N cells (256 per axis) of 4 slots (up to
 * 64 for cells of edge above 0.894 sigma), 16 bytes each, plus 4 bytes per
 * cell and per ion.  "Sweeps per launch" (MC_OPT_DA_SWEEPS) apply to it.    */
int mc_set_overlap_prefilter(mc_handle h, int chain, int W);

/* Training samples from the chain as it stands: for each ion i, the trial move
 * the chain would make next (sweep counter unchanged, nothing moves), the
 * features v above at the old and the trial position (v_pairs: N x 66, old
 * then trial), y = the exact pair sum sum_{j != i} q_j (1/r'_j - 1/r_j) minus
 * the tapered near-field part phi_near(x') - phi_near(x) (the part g must
 * learn: l_B q_i y is dE - dEt for g = 0), and
 * valid[i] = 1 unless the trial leaves the wall or overlaps.  Host buffers,
 * caller-owned.  Needs a surrogate set on the chain (its weights unused).  */
int mc_da_samples(mc_handle h, int chain, float *v_pairs, float *y, uint8_t *valid);

/* The surrogate MLP on the device (the project's own kernels; host buffers).
 * mc_mlp_forward: g at n points (v: n x 33).
 * mc_mlp_loss_grad: mean over n pairs of (g(v_trial) - g(v_old) - y)^2 and
 *   its gradient with respect to the 6401 parameters (FP32 arithmetic with the
 *   BF16 weights).
 * mc_mlp_train: Adam (beta 0.9/0.999, eps 1e-8) on FP32 master weights from
 *   w_init over `epochs` passes of mini-batches of `batch` pairs in the given
 *   order; the forward passes use the BF16-rounded weights; w_out gets the
 *   final BF16 weights and loss_per_epoch (nullable) each epoch's mean loss.  */
int mc_mlp_forward(const uint16_t *w_bf16, const float *v, int64_t n, float *g);
int mc_mlp_loss_grad(const uint16_t *w_bf16, const float *v_pairs, const float *y, int64_t n, double *loss,
                     float *grad);
int mc_mlp_train(const float *v_pairs, const float *y, int64_t n, const uint16_t *w_init, int epochs, int batch,
                 float lr, uint16_t *w_out, double *loss_per_epoch);

/* Total energy l_B sum_{i<j} q_i q_j / r_ij of n ions WITHOUT allocating
 * anything (no counterpart in the paper; an interface for callers that
 * cannot allocate device memory while they run: code being captured into a
 * CUDA graph, real-time loops that must not enter the allocator, hosts whose
 * device memory belongs to a pool they may not bypass).
 * pos_q_dev: device array of n float4 (x, y, z, valence), 16-byte aligned;
 * energy_dev: device double receiving the result; stream: a cudaStream_t as
 * void* (NULL = the default stream).  FP32 pair terms with FP64 row sums
 * (about 1e-7 of sum |q_i q_j| / r_ij; mc_energy's recomputed value uses
 * float-float terms and is about a million times closer).
 * The row sums live in one fixed device array of 1,048,576 doubles (8 MiB)
 * that the library's module carries on every GPU that loads it, until the
 * process exits; n > 1,048,576 returns MC_ERR_INVALID.  The first call on a
 * device looks up the array's address with that device current, and so does
 * the first call after the device's context was destroyed and created anew
 * (cudaDeviceReset), since the module may then sit at another address: make
 * that call before any stream capture (inside one it returns MC_ERR_INVALID
 * and enqueues nothing).  All calls share the array, so calls that
 * overlap on the GPU race; every call rewrites the rows it reads, so nothing
 * needs clearing.  The call only enqueues work on `stream`.                  */
int mc_total_energy_noalloc(const void *pos_q_dev, int64_t n, double l_B, double *energy_dev, void *stream);

/* Free all device and host memory of the handle. */
void mc_destroy(mc_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *mc_last_error(void);

/* Device information for roofline reporting: SM count, max SM clock (kHz). */
int mc_device_info(int *sm_count, int *sm_clock_khz, int *cc_major, int *cc_minor);

/* Test hook: Philox4x32-10 of the library's device code and of cuRAND's
 * curand_Philox4x32_10 for n (counter, key) pairs; ctr: n*4, key: n*2,
 * out_lib / out_curand: n*4 (all host arrays).                               */
int mc_test_philox(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out_lib, uint32_t *out_curand);

/* Measurement hook behind the ALU roofline (no counterpart in the paper):
 * the throughput of the two units the pair term uses, measured on the
 * current device.  Every thread runs 8 independent chains of one operation;
 * blocks of 256 threads, 1, 2, 4 and 8 of them per SM (8 to 64 resident
 * warps); clock64 around the loop.  rates (8 doubles, host): row w = 0..3
 * for 8 << w warps per SM, column 0 = rsqrt.approx.ftz per SM clock, column
 * 1 = FP32 operations per SM clock as packed fma.rn.f32x2 (two each).  Runs
 * synchronously on the default stream for about a millisecond.             */
int mc_unit_rates(double *rates);

/* Test hook: the library's device FP64 logarithm L(u) for n values. */
int mc_test_log(const double *u, int64_t n, double *out);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
