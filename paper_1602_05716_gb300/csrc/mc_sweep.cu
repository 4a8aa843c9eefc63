// mc_sweep.cu -- the persistent sweep kernel (sm_103a).
//
// What it computes is the sequential-updating Metropolis chain of Sec. 2:
// every sweep tries ions 0..N-1 in order; move i's energy change uses the
// current positions of all other ions (the Delta E_ij table of Sec. 2: ions
// j < i already at their outcome of this sweep, ions j > i at their position
// from the previous sweep).  How it computes it is GB300-specific:
//
//  * Work items are (chain, group of S = 128 consecutive ions, sweep),
//    handed out in stream order by an atomic ticket, so a CTA only ever waits
//    on work already claimed by a running CTA (no dependence on block
//    dispatch order, which the deadlock argument of Sec. 3.5 assumes).
//  * A group publishes its new positions into one of two buffers (sweep
//    parity) and then, per 32 ions, a release-stored word
//    ((sweep+1) << 32 | accept bits).  Readers acquire the word.  Tags only
//    grow, so no reset is needed (Algorithm 5's BlockState must be cleared).
//  * A CTA computes its S moves' pair sums against every other group's
//    published positions, tile by tile, oldest version first (the brush of
//    Algorithm 2), polling the next tiles' flags with relaxed loads and
//    prefetching their positions into registers.  Pairs with settled ions use
//    a cancellation-free FP32 form (error proportional to the displacement over
//    r^2), so the FP32 band stays narrow as N grows.
//  * The group just before this one (the "window") and this group's own
//    earlier moves (the lower triangle of Algorithms 3 and 4) are computed for
//    both possible positions of each such ion; the corrections
//    c_kj = term(trial_j) - term(old_j) stay in shared memory.  After the
//    window's accept bits arrive only masked sums remain; decisions are found
//    by interval rounds: a move whose outcome is the same for every
//    combination of still-unknown earlier outcomes is decided at once.
//  * A move is decided in FP32 only when its energy change lies outside a
//    proven FP32 error bound of the threshold; otherwise it is recomputed by
//    an accurate FP32 form (error proportional to the displacement), then in
//    double-single arithmetic, and finally in the oracle's FP64 arithmetic and
//    summation order, each tier with its own bound.
//  * The three groups before the window ("deep windows") are computed for
//    both positions too (on unless MC_OPT_DEEP_WINDOWS is 0).  Their
//    corrections live in tensor memory, written and read back with
//    tcgen05.st/ld, each warp in its own 32-lane quarter, so the last other
//    group a work item waits for is five groups back.
//  * Pairs mode (MC_OPT_PAIRS): a cluster of two CTAs shares one work item.
//    The helper sums every other tile and hands its sums over through a
//    global box, ordered by the cluster barriers.
//  * Barrier discipline: every __syncthreads sits under a CTA-uniform
//    condition.  A shared value that decides a branch containing barriers is
//    read by every thread before any thread may rewrite it, with a barrier in
//    between.  The resolve rounds put a barrier on both branches for this
//    reason: a warp that read a rewritten value once took the guard tiers'
//    barriers alone.
//  * Every wait is bounded by %globaltimer; on expiry the kernel records the
//    error, raises an abort flag and all CTAs return.
#include "mc_device.cuh"
#include "mc_da.cuh"

namespace mcg {

constexpr int MPT = 4;             // moves per thread in the pair loops
constexpr int TG = 4;              // groups per tile-ring buffer (one barrier per buffer)
constexpr int SL = T / (S / MPT);  // column slices (8)
constexpr int HALF = S / 2;
constexpr int DW = 3;              // deep windows: the groups g-2 .. g-1-DW, both positions, matrices in TMEM
static_assert(DW + 2 <= GB_SLOTS, "the guard board holds this group, the window and the deep windows");
constexpr unsigned TMEM_COLS = 512;  // power of two >= S * DW
static_assert(S == 128 && T == 256 && S * DW <= (int)TMEM_COLS && TMEM_COLS <= 512, "TMEM layout");

struct __align__(16) Smem {
    float4 own[S];    // this group: old positions (w = valence)
    float4 trial[S];  // this group: trial positions
    float4 wold[S];   // window group: old positions
    float4 wtri[S];   // window group: trial positions
    float4 dold[DW][S];  // deep windows (d = 0: the group before the window): old positions
    float4 dtri[DW][S];  // ... trial positions
    float4 tile[2][TG * S];  // tile ring: each buffer holds 1..TG consecutive groups
    float cin[S * CS];   // c[j][k], j < k, this group
    float cwin[S * CS];  // c[j][k], window ion j
    float bhi[S], blo[S];  // sum of terms with known positions (float-float)
    float kTs[S], kPs[S];      // far-field bound coefficients of each move (kTs < 0: not bounded, FP64 tier)
    float lo2ks[S], hi2ks[S];  // ... and its band of the overlap test on pair_far's squared distances
    float lo_w[S], hi_w[S], lo_i[S], hi_i[S];
    float Lf[S];   // -ln(u_acc) in FP32 (+inf if u_acc == 0)
    float bnd[S];  // static part of the FP32 band
    float wex[S];  // exact window correction (after the window's bits)
    float run[S];  // exact in-group correction over decided-accepted j < k
    float part[2][S];
    float wpart[2][S];
    float plo[2][S];
    float phi[2][S];
    float dE32[S];
    float dEt32[S];  // delayed acceptance: FP32 surrogate energy change
    float dEtB[S];   // ... its error bound (then the stage-2 part of the static band)
    double dEv[S];  // dE used for the ledger and the records
    double dEt64[S];  // delayed acceptance: the reference surrogate energy change, where computed
    unsigned ovo[S][WORDS], ovn[S][WORDS];    // x'_k overlaps old / trial position of in-group j < k
    unsigned wovo[S][WORDS], wovn[S][WORDS];  // ... of window ion j
    unsigned dovo[DW][S][WORDS], dovn[DW][S][WORDS];  // ... of deep-window ion j
    float wexd[S];  // deep windows: exact correction sums (their bits arrive before round 0)
    // deep-window pass, per (ion half, move slot): float-float sum of old-position terms, bound sums; after
    // the tiles: exact correction sums and overlap bits
    float dsh[2][S], dsl[2][S], dsA[2][S], dsT[2][S], dsC[2][S];
    float dlo[2][S], dhi[2][S];  // interval sums of deep window 0 (the group before the window: exact only at step 5)
    float dpart[2][S];
    unsigned dwo[2][S];
    float Qs[S], mind2[S];  // combined bound sum, minimum squared distance to a settled ion
    unsigned accw[WORDS], decw[WORDS], seen[WORDS], winacc[WORDS], acc0[WORDS], dec0[WORDS];
    unsigned d64w[WORDS];  // dEt64 known
    unsigned dacc[DW][WORDS];  // deep windows' accept bits
    unsigned tmem;             // TMEM base address (deep-window correction matrices)
    unsigned char st[S];
    signed char outcome[S];
    unsigned char tier[S];
    unsigned char pad0[S];
    unsigned char surv[S];  // moves that need pair sums (all moves of a plain chain; stage-1 survivors)
    unsigned char slot[S];  // inverse: move k's slot in surv (255: no pair sums)
    int damb[S];            // delayed acceptance: moves whose stage-1 decision needs the reference arithmetic
    double chunk[CHUNK];
    double redd[32];
    float redf[32];
    int ticket, ok, guard_k, ovl_flag;
    int hzs[2], tcnt[2];  // per buffer: publication horizon, groups staged
    int ns, namb;     // stage-1 survivors, ambiguous stage-1 moves
    int hcmd[2], hntl[2];  // helper warps: command and tile count of the hand-over, by its parity
};

// The helper warps' per-move tile sums (float-float, P, minimum squared distance), handed to the work-item warps
// between the tile pass and the slice combine.  They alias part and wpart, which are first written after it.
__device__ __forceinline__ float *help_h(Smem &sm) { return sm.part[0]; }
__device__ __forceinline__ float *help_l(Smem &sm) { return sm.part[1]; }
__device__ __forceinline__ float *help_p(Smem &sm) { return sm.wpart[0]; }
__device__ __forceinline__ float *help_m(Smem &sm) { return sm.wpart[1]; }

// More than half of an SM's 228 KB of shared memory: one CTA per SM, so each CTA's TMEM allocation (at most
// 512 columns) is granted at once and never waits for another CTA.
static_assert(sizeof(Smem) > 116 * 1024, "one CTA per SM");

// Tensor memory (TMEM) holds the deep-window correction matrices: lane = move slot, column = S d + j for ion j of
// deep window d.  tcgen05 loads and stores of shape 32x32b move one lane per thread; warp w reaches lanes
// [32 (w mod 4), 32 (w mod 4) + 32), so each warp only touches its own lane quarter and column half.
__device__ __forceinline__ void tmem_alloc(unsigned *dst)  // one whole warp
{
    __syncwarp();  // .aligned: the whole warp, converged
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "r"(TMEM_COLS)
                 : "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr)  // one whole warp
{
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

__device__ __forceinline__ void tmem_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 16 consecutive columns of this thread's lane (whole warp, converged).  The store reads its source registers
// asynchronously, so it waits for its completion in the same statement: no later instruction may overwrite
// those registers before the tensor memory holds their values.
__device__ __forceinline__ void tmem_st16(unsigned taddr, const float (&v)[16])
{
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};\n"
        "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st()
{
    __syncwarp();
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Load and wait in one statement, so that no use of the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16])
{
    __syncwarp();
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Thread-block cluster of two (pairs mode): rank and a full barrier of both CTAs with release/acquire order
// (the hand-over goes through global memory, so nothing reads a partner's shared memory).
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    __syncwarp();  // .aligned: every warp converged (callers follow single-lane branches)
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// 32 consecutive columns of this thread's lane, load and wait in one statement.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32])
{
    __syncwarp();
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr unsigned ST_WALL = 1u, ST_UZERO = 2u, ST_INACTIVE = 4u, ST_OVL_CERTAIN = 8u, ST_OVL_AMBIG = 16u,
                   ST_OVL_POSSIBLE = 32u, ST_DA_DONE = 64u;
constexpr int OUT_INACTIVE = 15;  // padding slot of a ragged group (never recorded or counted)
constexpr unsigned FULL = 0xffffffffu;

// Bound constants (units of u = 2^-24) of the FP32 band: per pair term of the direct form, FP32 partial sums of
// <= 16 terms promoted exactly by TwoSum, and the FP32 sums and interval sums of <= S corrections.
constexpr float C_TERM = 10.0f;           // per-term error of q_j (1/r' - 1/r) relative to |q_j| (1/r' + 1/r)
                                          // (both-position ions, direct form)
constexpr float C_SUM = 24.0f;            // FP32 partials of <= 16 terms, TwoSum-accumulated
constexpr float C_CORR = 2.0f * (S + 8);  // FP32 sums and interval sums of <= S corrections

__device__ __forceinline__ float finf()
{
    return __int_as_float(0x7f800000);
}

__device__ __forceinline__ bool bit(const unsigned *w, int j)
{
    return (w[j >> 5] >> (j & 31)) & 1u;
}

// Mask of the bits j < k within word w.
__device__ __forceinline__ unsigned below(int k, int w)
{
    return (w * 32 + 32 <= k) ? 0xffffffffu : (w * 32 >= k ? 0u : ((1u << (k - w * 32)) - 1u));
}

// Barriers.  Barrier 1 spans the T threads that run the work items: every barrier of the work-item code.  In the
// kernel with helper warps (2T threads), barrier 2 spans those and the helpers during the tile pass, and barrier 0
// the whole CTA at start and exit.
__device__ __forceinline__ void bar_main()
{
    asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
}

__device__ __forceinline__ void bar_all()
{
    asm volatile("bar.sync 2, %0;" ::"n"(2 * T) : "memory");
}

// Tile-pass hand-over to the helper warps (Smem::hcmd).
constexpr int HC_SKIP = 0, HC_RUN = 1, HC_EXIT = 2;

// ---------------------------------------------------------------------------
// The shared guard (Ctl::gb).  Tiers 2 and 3 of a move sum N terms; while one work item decides its group, most
// of the launch's work items wait for that group's outcome.  So a work item whose move needs tier 2 or 3 posts
// the move on the board, and its own warps take chunks of GB_CHUNK partners together with every warp that waits
// in wait_words meanwhile.  Per chunk: the tier's own per-pair terms and error bounds, summed per lane
// (compensated, as in the tier) and over the warp in FP64.  The poster adds the chunk sums in chunk order with a
// compensated FP64 sum, so the sum and the bound are the tier's up to FP64 roundings far inside the tier's margin,
// and the decision rule is the tier's.  One request at a time: a work item that finds the board taken (another
// chain of a batch) runs the tier on its own CTA, and so does every work item after a wait on the board gave up.

__device__ __forceinline__ unsigned ld_acquire32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Warp: take chunks of the posted request until none is left (defined with the guard tiers).
__device__ __noinline__ void gb_help(Ctl *ctl);

// Is a posted request waiting for warps?  (Every lane gets the answer.)
__device__ __forceinline__ bool gb_open(Ctl *ctl)
{
    int w = 0;
    if ((threadIdx.x & 31) == 0 && ctl->gb) {
        const unsigned long long v = ld_relaxed(&ctl->gnext);
        w = ((unsigned)v & 0xffffu) < (((unsigned)(v >> 16)) & 0xffffu);
    }
    return __shfl_sync(FULL, w, 0) != 0;
}

// Warp 0 waits until the sweep tags of the nw words of group J lie in [lo, hi]
// (acquire).  Returns false on timeout, protocol error or abort.  bits (lane w)
// gets word w's accept bits.
__device__ bool wait_words(const ChainDev &ch, int J, int nw, unsigned lo, unsigned hi, Ctl *ctl, unsigned &bits,
                           bool sleep = true, bool outcome_words = false, bool help = false)
{
    const unsigned long long *words = outcome_words ? ch.bits : ch.flags;
    const int lane = threadIdx.x & 31;
    unsigned long long t0 = 0;  // the clock starts at the first check, so a wait that succeeds at once reads none
    unsigned spins = 0;
    bool done = lane >= nw;
    bits = 0u;
    for (;;) {
        if (!done) {
            const unsigned long long v = outcome_words ? ld_relaxed(&words[J * WORDS + lane])
                                                       : ld_acquire(&words[J * WORDS + lane]);
            const unsigned tag = (unsigned)(v >> 32);
            if ((int)(tag - lo) >= 0 && (int)(hi - tag) >= 0) {
                done = true;
                bits = (unsigned)v;
            } else if ((int)(tag - hi) > 0) {
                atomicCAS(&ctl->err, 0, KERR_PROTOCOL);
                atomicExch(&ctl->abort, 1);
            }
        }
        if (__all_sync(FULL, done)) return true;
        ++spins;
        if (help && (spins & 7) == 0 && gb_open(ctl)) gb_help(ctl);
        if (spins > 16 && sleep) __nanosleep(32);
        if ((spins & 31) == 0 && *(volatile int *)&ctl->abort) return false;
        if ((spins & 63) == 0) {
            const unsigned long long now = __shfl_sync(FULL, globaltimer(), 0);
            if (t0 == 0) t0 = now;
            else if ((long long)(now - t0) > ctl->timeout_ns) {
                if (lane == 0) {
                    if (atomicCAS(&ctl->err, 0, KERR_TIMEOUT) == 0) ctl->err_info = ((unsigned long long)J << 32) | lo;
                    atomicExch(&ctl->abort, 1);
                }
                __syncwarp();
                return false;
            }
        }
    }
}

// Bound coefficients of the tiles' pair form (pair_far2) for a move of length at most dn when every settled ion
// is at least sp from both the old and the trial position (x = dn / sp).  Following tier 2's per-term bound with
// Ro <= Rn + dn and rho >= (1 - x/2) min(Rn, Ro):
//   per term  |err| <= u |q| (kT |t| + kP rn ro),   kT = kD + 20,  kP = (6 (1 + x/2) + k3) dn,
//   kD = 3 (1+x)^2 + 4 (2x + x^2) + 8x^2 + 1,   k3 = (1+x) (3/g^2 + 2x/g^3),  g = 1 - x/2;
// the squared distance Dn is within u kO max(Dn, sigma^2) of |a - y|^2, kO = 5 (1+x)^2 + 14x + 16x^2 + 1.
// pair_far2's three-FMA Dd is within 6u dn (Ro + dn), where tier 2's dot product is within 4u M <= 4u dn (Rn + Ro).
// Relative to Dn that is at most u (6x + 12x^2) against u (8x + 4x^2): the 8x^2 added to kD and kO.  Through t's
// factor (rn ro)^2 / (rn + ro) it is at most 6u (1 + x/2) dn rn ro against 4u dn rn ro: kP's 6 (1 + x/2).
// Returns false for x >= 1.75, where the move is left to the FP64 tier.
__device__ __forceinline__ bool far_coeffs(float dn, float sp, float &kT, float &kP, float &kO)
{
    const float x = dn / sp * (1.0f + 0x1p-20f);
    if (!(x < 1.75f)) return false;
    const float x1 = 1.0f + x, g = 1.0f - 0.5f * x;
    const float kD = 3.0f * x1 * x1 + 4.0f * x * (2.0f + x) + 8.0f * x * x + 1.0f;
    const float k3 = x1 * (3.0f / (g * g) + 2.0f * x / (g * g * g));
    kT = (kD + 20.0f) * (1.0f + 0x1p-10f);
    kP = (6.0f * (1.0f + 0.5f * x) + k3) * dn * (1.0f + 0x1p-10f);
    kO = (5.0f * x1 * x1 + x * (14.0f + 16.0f * x) + 1.0f) * (1.0f + 0x1p-4f);
    return true;
}

__device__ __forceinline__ float pair_term(const float4 a, const float4 b, const float4 y, float &Ay, float &d2n)
{
    const float dxn = a.x - y.x, dyn = a.y - y.y, dzn = a.z - y.z;
    d2n = fmaf(dzn, dzn, fmaf(dyn, dyn, dxn * dxn));
    const float dxo = b.x - y.x, dyo = b.y - y.y, dzo = b.z - y.z;
    const float d2o = fmaf(dzo, dzo, fmaf(dyo, dyo, dxo * dxo));
    const float rn = rsqrt_approx(d2n), ro = rsqrt_approx(d2o);
    Ay = fabsf(y.w) * (rn + ro);
    return y.w * (rn - ro);
}

// Exact overlap test |a - y|^2 < sigma^2 from the FP32 squared distance, the
// FP64 squared distance of the FP32 points deciding inside the band.
__device__ __forceinline__ bool overlaps(float d2f, const float4 a, const float4 y, float lo, float hi, double sig2)
{
    if (d2f < lo) return true;
    if (d2f > hi) return false;
    return d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < sig2;
}

// Both-position pair of move k against an ion j whose outcome is unknown
// (an earlier ion of this group, or an ion of the window group).
__device__ __forceinline__ void both_pair(float *cm, unsigned (*ovo)[WORDS], unsigned (*ovn)[WORDS], int k, int j,
                                          const float4 a, const float4 b, const float4 yo, const float4 yn, float &s,
                                          float &A, float &Tt, float &TC, float lo, float hi, double sig2)
{
    float Ao, An, d2o_n, d2n_n;
    const float to = pair_term(a, b, yo, Ao, d2o_n);
    const float tn = pair_term(a, b, yn, An, d2n_n);
    s += to;
    Tt += fabsf(to);
    A += Ao + An;
    const float c = tn - to;
    cm[j * CS + k] = c;
    TC += fabsf(c);
    if (overlaps(d2o_n, a, yo, lo, hi, sig2)) atomicOr(&ovo[k][j >> 5], 1u << (j & 31));
    if (overlaps(d2n_n, a, yn, lo, hi, sig2)) atomicOr(&ovn[k][j >> 5], 1u << (j & 31));
}

// Both-position pair for the second window: as both_pair, returning the correction instead of storing it.
__device__ __forceinline__ float both_pair_c(unsigned (*ovo)[WORDS], unsigned (*ovn)[WORDS], int k, int j, const float4 a,
                                             const float4 b, const float4 yo, const float4 yn, float &s, float &A,
                                             float &Tt, float &TC, float lo, float hi, double sig2)
{
    float Ao, An, d2o_n, d2n_n;
    const float to = pair_term(a, b, yo, Ao, d2o_n);
    const float tn = pair_term(a, b, yn, An, d2n_n);
    s += to;
    Tt += fabsf(to);
    A += Ao + An;
    const float c = tn - to;
    TC += fabsf(c);
    if (overlaps(d2o_n, a, yo, lo, hi, sig2)) atomicOr(&ovo[k][j >> 5], 1u << (j & 31));
    if (overlaps(d2n_n, a, yn, lo, hi, sig2)) atomicOr(&ovn[k][j >> 5], 1u << (j & 31));
    return c;
}

struct Ctx {
    const ChainDev *ch;
    const float4 *Pprev;  // positions after sweep s-1
    const float4 *Pcur;   // positions after sweep s (groups < g published)
    int N, B, g, k0, nk, Jw, nwk, nd;  // nd deep windows: groups g-2 .. g-1-nd
    bool win;
    unsigned long long s;
};

// Position of ion j as seen by move k of this group (all earlier moves of the
// group decided, the window's bits known).
__device__ __forceinline__ float4 position_of(const Smem &sm, const Ctx &c, int k, int j)
{
    const int J = j / S, l = j - J * S;
    if (J == c.g) return (l < k && bit(sm.accw, l)) ? sm.trial[l] : sm.own[l];
    if (c.win && J == c.Jw) return bit(sm.winacc, l) ? sm.wtri[l] : sm.wold[l];
    const int d = c.g - 2 - J;
    if (J < c.g && d >= 0 && d < c.nd) return bit(sm.dacc[d], l) ? sm.dtri[d][l] : sm.dold[d][l];
    return J > c.g ? __ldcg(&c.Pprev[j]) : __ldcg(&c.Pcur[j]);
}

// Guard tiers stage the positions seen by move k in blocks of GSTAGE ions,
// reusing the window-correction matrix (dead once the window's sums are
// formed): branch-free 16-byte loads of every ion's published position, then
// this group's and the window group's ions patched from shared memory.  The
// callers skip ion k itself and the padding beyond N by index.
constexpr int GSTAGE = 2048;
static_assert(GSTAGE * 16 + GSTAGE * 8 <= S * CS * 4, "guard staging fits in the window matrix");

__device__ __forceinline__ float4 *stage_buf(Smem &sm)
{
    return reinterpret_cast<float4 *>(sm.cwin);
}

__device__ __forceinline__ double *stage_terms(Smem &sm)
{
    return reinterpret_cast<double *>(reinterpret_cast<float4 *>(sm.cwin) + GSTAGE);
}

__device__ void stage_positions(Smem &sm, const Ctx &c, int k, int j0)
{
    float4 *buf = stage_buf(sm);
    const int tid = threadIdx.x;
    bar_main();
#pragma unroll
    for (int u = 0; u < GSTAGE / T; ++u) {
        const int t = u * T + tid, j = j0 + t;
        const float4 *src = ((j >> 7) > c.g) ? c.Pprev : c.Pcur;
        buf[t] = (j < c.N) ? __ldcg(&src[j]) : make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
    }
    bar_main();
    if (tid < S) {
        const int l = tid;
        int t = c.k0 + l - j0;
        if (t >= 0 && t < GSTAGE && l < c.nk) {
            buf[t] = (l < k && bit(sm.accw, l)) ? sm.trial[l] : sm.own[l];
        }
        if (c.win && l < c.nwk) {
            t = c.Jw * S + l - j0;
            if (t >= 0 && t < GSTAGE) buf[t] = bit(sm.winacc, l) ? sm.wtri[l] : sm.wold[l];
        }
        for (int d = 0; d < c.nd; ++d) {
            t = (c.g - 2 - d) * S + l - j0;
            if (t >= 0 && t < GSTAGE) buf[t] = bit(sm.dacc[d], l) ? sm.dtri[d][l] : sm.dold[d][l];
        }
    }
    bar_main();
}

// Sum of per-thread FP64 values and FP32 bound terms over the CTA (thread 0 gets it).
__device__ __forceinline__ void block_sum(Smem &sm, double v, float bb, double &tot, double &btot)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(FULL, v, o);
        bb += __shfl_xor_sync(FULL, bb, o);
    }
    if ((tid & 31) == 0) {
        sm.redd[tid >> 5] = v;
        sm.redf[tid >> 5] = bb;
    }
    bar_main();
    tot = 0.0;
    btot = 0.0;
    if (tid == 0)
        for (int w = 0; w < T / 32; ++w) {
            tot += sm.redd[w];
            btot += (double)sm.redf[w];
        }
}

// ---------------------------------------------------------------------------
// Guard tiers for move k (whole CTA).  Return 0 accept, 1 reject, -1 undecided.

// Tier 2: accurate FP32.  With e = y - b and delta = a - b the pair's energy
// change is q (delta . (2e - delta)) (rn ro)^2 / (rn + ro): no difference of
// two large inverse distances, so the rounding error scales with
// |delta| / r^2 instead of 1/r.  Per-term bound:
// |q| [ |t| (rel(Dn) + 19u) + 4u M (rn ro)^2/(rn+ro) + u |delta| (2 Ro + rho)/rho^3 ]
// with rho a lower bound of the distance from y to the segment [b, a].
constexpr double T2_KB = 1.25, T2_KR = 0x1p-40, T3_KB = 1.01 * 0x1p-38, T3_KR = 0x1p-48;

// A guard tier's outcome: dE = lq tot against the threshold L64 with the margin kb |lq| bt (bt the sum of the
// terms' error bounds) plus kr (|dE| + |L64|) for the final roundings and xs: 0 accept, 1 reject, -1 undecided.
__device__ __forceinline__ int guard_outcome(double lq, double tot, double bt, double kb, double kr, double L64,
                                             double xs, double &dE)
{
    dE = lq * tot;
    const double Bm = fabs(lq) * bt * kb + kr * (fabs(dE) + fabs(L64)) + xs + 1e-300;
    return (dE < L64 - Bm) ? 0 : ((dE > L64 + Bm) ? 1 : -1);
}

// Tier 2's term for partner y (old position b, displacement (dx, dy, dz) of length at most dn, rho0 the
// smallest distance from a partner to the segment [b, a] that the overlap rule allows) added to the compensated
// sum (hi, lo), and its error bound to bsum.
__device__ __forceinline__ void t2_pair(const float4 b, float dx, float dy, float dz, float dn, float rho0,
                                        const float4 y, float &hi, float &lo, float &bsum)
{
    const float ex = y.x - b.x, ey = y.y - b.y, ez = y.z - b.z;
    const float Do = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
    const float wx = fmaf(2.0f, ex, -dx), wy = fmaf(2.0f, ey, -dy), wz = fmaf(2.0f, ez, -dz);
    const float Dd = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
    const float M = fabsf(dx * wx) + fabsf(dy * wy) + fabsf(dz * wz);
    const float Dn = Do - Dd;
    const float ro = rsqrt_approx(Do), rn = rsqrt_approx(Dn);
    const float pr = rn * ro, inv = rcp_approx(rn + ro);
    const float t = Dd * pr * pr * inv;
    const float term = y.w * t;
    float e, s;
    two_sum(hi, term, s, e);
    hi = s;
    lo += e;
    const float relDn = fmaf(3.0f * U32, Do, 4.0f * U32 * M) * rn * rn + U32;
    const float Ro = Do * ro * (1.0f + 0x1p-18f), Rn = Dn * rn;
    const float rho = fmaxf(fminf(Rn, Ro) * (1.0f - 0x1p-18f) - 0.5f * dn, rho0);
    const float ir = rcp_approx(rho);
    const float E1 = fabsf(t) * (relDn + 19.0f * U32);
    const float E2 = 4.0f * U32 * M * pr * pr * inv;
    const float E3 = U32 * dn * (2.0f * Ro + rho) * ir * ir * ir;
    bsum += fabsf(y.w) * (E1 + E2 + E3);
}

__device__ int tier2(Smem &sm, const Ctx &c, int k, double L64, double xs, double &dE_out)
{
    const int tid = threadIdx.x;
    const float4 a = sm.trial[k], b = sm.own[k];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float dn = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) * (1.0f + 0x1p-18f);
    const float s2 = (float)c.ch->sig2;
    const float rho0 = sqrtf(fmaxf(s2 * (1.0f - 0x1p-18f) - 0.25f * dn * dn, 0.0f)) * (1.0f - 0x1p-18f);
    const int i = c.k0 + k;
    float hi = 0.f, lo = 0.f, bsum = 0.f;
    const float4 *buf = stage_buf(sm);
    for (int j0 = 0; j0 < c.N; j0 += GSTAGE) {
      stage_positions(sm, c, k, j0);
#pragma unroll 2
      for (int u = 0; u < GSTAGE / T; ++u) {
        const int j = j0 + u * T + tid;
        if (j >= c.N || j == i) continue;
        t2_pair(b, dx, dy, dz, dn, rho0, buf[u * T + tid], hi, lo, bsum);
      }
    }
    double tot, bt;
    block_sum(sm, (double)hi + (double)lo, bsum, tot, bt);
    if (tid == 0) {
        double dE;
        sm.guard_k = guard_outcome(c.ch->lB * (double)a.w, tot, bt, T2_KB, T2_KR, L64, xs, dE);
        sm.redd[16] = dE;
    }
    bar_main();
    const int out = sm.guard_k;
    dE_out = sm.redd[16];
    bar_main();
    return out;
}

// Double-single arithmetic for tier 3 (each value is an unevaluated sum hi + lo).
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e = e + (al + bl);
    sh = s + e;
    sl = e - (sh - s);
}

__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    float p, e;
    two_prod(ah, bh, p, e);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    ph = p + e;
    pl = e - (ph - p);
}

// 1/sqrt(D) for D = (dh, dl) in double-single: FP32 seed, one Newton step with
// the residual 1 - D r^2 formed in double-single.
__device__ __forceinline__ void df_rsqrt(float dh, float dl, float &rh, float &rl)
{
    const float r0 = rsqrt_approx(dh);
    float ph, pl, xh, xl;
    two_prod(r0, r0, ph, pl);
    df_mul(dh, dl, ph, pl, xh, xl);
    const float res = (1.0f - xh) - xl;
    const float corr = 0.5f * r0 * res;
    rh = r0 + corr;
    rl = corr - (rh - r0);
}

// Tier 3's term for partner y in double-single, added to (hh, hl); |q_y| (1/r' + 1/r) added to absum.
__device__ __forceinline__ void t3_pair(const float4 a, const float4 b, const float4 y, float &hh, float &hl,
                                        float &absum)
{
    float Dn_h = 0.f, Dn_l = 0.f, Do_h = 0.f, Do_l = 0.f;
    const float av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z}, yv[3] = {y.x, y.y, y.z};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float eh, el, sh, sl;
        two_sum(av[q], -yv[q], eh, el);  // exact a - y
        df_mul(eh, el, eh, el, sh, sl);
        df_add(Dn_h, Dn_l, sh, sl, Dn_h, Dn_l);
        two_sum(bv[q], -yv[q], eh, el);  // exact b - y
        df_mul(eh, el, eh, el, sh, sl);
        df_add(Do_h, Do_l, sh, sl, Do_h, Do_l);
    }
    float rnh, rnl, roh, rol, th, tl, qh, ql;
    df_rsqrt(Dn_h, Dn_l, rnh, rnl);
    df_rsqrt(Do_h, Do_l, roh, rol);
    df_add(rnh, rnl, -roh, -rol, th, tl);
    df_mul(th, tl, y.w, 0.0f, qh, ql);
    df_add(hh, hl, qh, ql, hh, hl);
    absum += fabsf(y.w) * (rnh + roh);
}

// One chunk of the posted request (whole warp); lane 0 stores the chunk's sums.  The request is read through L2:
// it was written by another SM after this SM may have cached an older one.  A waiting warp often runs alone on
// its SM, so the positions are loaded GQ ions per lane ahead of their use.
constexpr int GQ = 4;
__device__ __forceinline__ void gb_chunk(GuardBoard *gb, int q)
{
    const int lane = threadIdx.x & 31;
    const int tier = __ldcg(&gb->tier), N = __ldcg(&gb->N), g = __ldcg(&gb->g), i = __ldcg(&gb->i);
    const float4 a = __ldcg(&gb->a), b = __ldcg(&gb->b);
    const float4 *Pp = (const float4 *)__ldcg((const unsigned long long *)&gb->Pprev);
    const float4 *Pc = (const float4 *)__ldcg((const unsigned long long *)&gb->Pcur);
    int sJ[GB_SLOTS];
#pragma unroll
    for (int u = 0; u < GB_SLOTS; ++u) sJ[u] = __ldcg(&gb->slotJ[u]);
    const int j0 = q * GB_CHUNK, j1 = min(N, j0 + GB_CHUNK);
    // the address of partner j's position: the request's copy for the groups it holds, else the published arrays
    auto src = [&](int j) -> const float4 * {
        const int J = j / S;
        const float4 *p = &(J > g ? Pp : Pc)[j];
#pragma unroll
        for (int u = GB_SLOTS - 1; u >= 0; --u)
            if (sJ[u] == J) p = &gb->ovl[u][j - J * S];
        return p;
    };
    auto fetch = [&](float4(&dst)[GQ], int base) {
#pragma unroll
        for (int u = 0; u < GQ; ++u) {
            const int j = base + 32 * u;
            dst[u] = (j < j1) ? __ldcg(src(j)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    // two batches of GQ partners per lane: one in flight while the other is summed
    auto sweep2 = [&](auto &&sum8) {
        float4 yA[GQ], yB[GQ];
        fetch(yA, j0 + lane);
        for (int base = j0 + lane; base < j1; base += 64 * GQ) {
            const int bB = base + 32 * GQ;
            if (bB < j1) fetch(yB, bB);
            sum8(yA, base);
            if (bB < j1) {
                if (bB + 32 * GQ < j1) fetch(yA, bB + 32 * GQ);
                sum8(yB, bB);
            }
        }
    };
    double v;
    float bb;
    if (tier == 2) {
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const float dn = __ldcg(&gb->dn), rho0 = __ldcg(&gb->rho0);
        float hi = 0.f, lo = 0.f, bsum = 0.f;
        sweep2([&](const float4(&yy)[GQ], int base) {
#pragma unroll
            for (int u = 0; u < GQ; ++u) {
                const int j = base + 32 * u;
                if (j < j1 && j != i) t2_pair(b, dx, dy, dz, dn, rho0, yy[u], hi, lo, bsum);
            }
        });
        v = (double)hi + (double)lo;
        bb = bsum;
    } else {
        float hh = 0.f, hl = 0.f, absum = 0.f;
        sweep2([&](const float4(&yy)[GQ], int base) {
#pragma unroll
            for (int u = 0; u < GQ; ++u) {
                const int j = base + 32 * u;
                if (j < j1 && j != i) t3_pair(a, b, yy[u], hh, hl, absum);
            }
        });
        v = (double)hh + (double)hl;
        bb = absum;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(FULL, v, o);
        bb += __shfl_xor_sync(FULL, bb, o);
    }
    if (lane == 0) {
        gb->part[q] = v;
        gb->bpart[q] = (double)bb;
    }
}

// A warp takes a chunk is taken by a compare-and-swap on the
// whole (request, chunks, next) word, so a warp that read an older request takes nothing from a newer one.
__device__ __noinline__ void gb_help(Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long v = 0;
        int got = 0;
        if (lane == 0) {
            v = ld_relaxed(&ctl->gnext);
            for (int tries = 0; tries < 4096; ++tries) {  // every failed swap is another warp's progress
                const unsigned n = (unsigned)(v >> 16) & 0xffffu, nx = (unsigned)v & 0xffffu;
                if (nx >= n) break;
                const unsigned long long w = atomicCAS(&ctl->gnext, v, v + 1ull);
                if (w == v) {
                    got = 1;
                    break;
                }
                v = w;
            }
        }
        if (!__shfl_sync(FULL, got, 0)) return;
        v = __shfl_sync(FULL, v, 0);
        fence_acq_rel();  // the request was written before it was posted
        gb_chunk(ctl->gb, (int)(v & 0xffffull));
        __syncwarp();
        if (lane == 0) {
            fence_acq_rel();  // the chunk's sums before its count
            atomicAdd(&ctl->gdone, 1u);
        }
        __syncwarp();
    }
}

// Tier 3: every pair term in double-single arithmetic (distances from exact
// FP32 differences); bound 2^-38 l_B |q_i| sum_j |q_j| (1/r' + 1/r).
__device__ int tier3(Smem &sm, const Ctx &c, int k, double L64, double xs, double &dE_out)
{
    const int tid = threadIdx.x;
    const float4 a = sm.trial[k], b = sm.own[k];
    const int i = c.k0 + k;
    float hh = 0.f, hl = 0.f, absum = 0.f;
    const float4 *buf = stage_buf(sm);
    for (int j0 = 0; j0 < c.N; j0 += GSTAGE) {
      stage_positions(sm, c, k, j0);
      for (int u = 0; u < GSTAGE / T; ++u) {
        const int j = j0 + u * T + tid;
        if (j >= c.N || j == i) continue;
        t3_pair(a, b, buf[u * T + tid], hh, hl, absum);
      }
    }
    double tot, bt;
    block_sum(sm, (double)hh + (double)hl, absum, tot, bt);
    if (tid == 0) {
        double dE;
        sm.guard_k = guard_outcome(c.ch->lB * (double)a.w, tot, bt, T3_KB, T3_KR, L64, xs, dE);
        sm.redd[16] = dE;
    }
    bar_main();
    const int out = sm.guard_k;
    dE_out = sm.redd[16];
    bar_main();
    return out;
}

// Tier 2 or 3 of move k through the board (whole CTA).  Returns 0 accept, 1 reject, -1 undecided, or -2 when
// the board is taken (the caller runs the tier on its own CTA).  The request holds the positions the move sees
// from shared memory: its own group (moves before k decided), the window and the deep windows.
__device__ int gb_tier(Smem &sm, const Ctx &c, Ctl *ctl, int k, int tier, double L64, double xs, double &dE_out)
{
    const int tid = threadIdx.x;
    GuardBoard *gb = ctl->gb;
    const unsigned n = (unsigned)((c.N + GB_CHUNK - 1) / GB_CHUNK);
    if (tid == 0) sm.guard_k = (gb && n <= 0xffffu && atomicCAS(&ctl->glock, 0u, 1u) == 0u) ? 1 : 0;
    bar_main();
    const bool mine = sm.guard_k != 0;
    bar_main();
    if (!mine) return -2;
    const float4 a = sm.trial[k], b = sm.own[k];
    for (int q = tid; q < GB_SLOTS * S; q += T) {
        const int u = q / S, l = q - u * S;
        int J = -1;
        if (u == 0) J = c.g;
        else if (u == 1) J = c.win ? c.Jw : -1;
        else if (u - 2 < c.nd) J = c.g - u;  // deep window u - 2: group g - 2 - (u - 2)
        gb->ovl[u][l] = (J >= 0) ? position_of(sm, c, k, J * S + l) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (l == 0) gb->slotJ[u] = J;
    }
    if (tid == 0) {
        gb->tier = tier;
        gb->N = c.N;
        gb->g = c.g;
        gb->i = c.k0 + k;
        gb->a = a;
        gb->b = b;
        gb->Pprev = c.Pprev;
        gb->Pcur = c.Pcur;
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const float dn = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) * (1.0f + 0x1p-18f);
        const float s2 = (float)c.ch->sig2;
        gb->dn = dn;
        gb->rho0 = sqrtf(fmaxf(s2 * (1.0f - 0x1p-18f) - 0.25f * dn * dn, 0.0f)) * (1.0f - 0x1p-18f);
    }
    fence_acq_rel();
    bar_main();
    if (tid == 0) {
        atomicExch(&ctl->gdone, 0u);
        const unsigned long long id = (ld_relaxed(&ctl->gnext) >> 32) + 1ull;
        fence_acq_rel();
        atomicExch(&ctl->gnext, (id << 32) | ((unsigned long long)n << 16));
    }
    bar_main();
    gb_help(ctl);  // this work item's warps take chunks too
    if (tid == 0) {
        // the chunks taken by other warps: each is a bounded computation
        bool ok = true;
        unsigned long long t0 = 0;
        for (unsigned spins = 1; ld_acquire32(&ctl->gdone) < n; ++spins) {
            if ((spins & 63) == 0) {
                const unsigned long long now = globaltimer();
                if (t0 == 0) t0 = now;
                else if ((long long)(now - t0) > ctl->timeout_ns) {
                    ok = false;
                    break;
                }
            }
        }
        int out = -1;
        double dE = 0.0;
        if (ok) {
            double sh = 0.0, sl = 0.0, bt = 0.0;
            for (unsigned q = 0; q < n; ++q) {  // compensated, in chunk order
                const double p = __ldcg(&gb->part[q]);
                const double t = sh + p, bp = t - sh;
                sl += (sh - (t - bp)) + (p - bp);
                sh = t;
                bt += __ldcg(&gb->bpart[q]);
            }
            out = guard_outcome(c.ch->lB * (double)a.w, sh + sl, bt, tier == 2 ? T2_KB : T3_KB,
                                tier == 2 ? T2_KR : T3_KR, L64, xs, dE);
            fence_acq_rel();
            atomicExch(&ctl->glock, 0u);
        } else {
            // a chunk never arrived: the board stays taken (its late writes land on no newer request), the launch
            // ends with the error, and this move goes on to tier 4
            if (atomicCAS(&ctl->err, 0, KERR_TIMEOUT) == 0) ctl->err_info = 0xffffffffull;
            atomicExch(&ctl->abort, 1);
        }
        sm.guard_k = out;
        sm.redd[16] = dE;
    }
    bar_main();
    const int out = sm.guard_k;
    dE_out = sm.redd[16];
    bar_main();
    return out;
}

// Tier 4: the oracle's arithmetic -- FP64 terms with IEEE sqrt and division,
// summed sequentially within 1024-index chunks, chunk sums added in order;
// overlap from the FP64 squared distance.
__device__ void tier4(Smem &sm, const Ctx &c, int k, double &dE_out, bool &ovl_out)
{
    const int tid = threadIdx.x;
    const int N = c.N;
    const int i = c.k0 + k;
    const float4 a = sm.trial[k], b = sm.own[k];
    const float4 *buf = stage_buf(sm);
    double *terms = stage_terms(sm);
    if (tid == 0) sm.ovl_flag = 0;
    double total = 0.0;
    for (int j0 = 0; j0 < N; j0 += GSTAGE) {
        stage_positions(sm, c, k, j0);
        for (int u = 0; u < GSTAGE / T; ++u) {
            const int t = u * T + tid;
            const int j = j0 + t;
            const float4 y = buf[t];
            double v = 0.0;
            if (j < N && j != i) {
                bool o;
                v = term_fp64(a, b, y, o, c.ch->sig2);
                if (o) sm.ovl_flag = 1;
            }
            terms[t] = v;
        }
        bar_main();
        // each 1024-ion chunk is summed sequentially by its own thread (chunks are independent)
        if (tid < GSTAGE / CHUNK) {
            const int cb = j0 + tid * CHUNK;
            double s = 0.0;
            if (cb < N) {
                const int len = min(CHUNK, N - cb);
                for (int jj = 0; jj < len; ++jj)
                    if (cb + jj != i) s = __dadd_rn(s, terms[tid * CHUNK + jj]);
            }
            sm.redd[tid] = s;
        }
        bar_main();
        if (tid == 0)
            for (int q = 0; q < GSTAGE / CHUNK; ++q)
                if (j0 + q * CHUNK < N) total = __dadd_rn(total, sm.redd[q]);
    }
    bar_main();
    if (tid == 0) sm.redd[16] = __dmul_rn(__dmul_rn(c.ch->lB, (double)a.w), total);
    bar_main();
    dE_out = sm.redd[16];
    ovl_out = sm.ovl_flag != 0;
    bar_main();
}

// Exact overlap test of move k's trial position against every other ion as move k sees it (all earlier
// moves of the group decided): an FP32 prefilter (its squared distance errs by at most 5u, far inside
// 2^-12), then the oracle's FP64 squared distance for the few ions it lets through.  Settles a move whose
// FP32 minimum fell inside the overlap band at the cost of one pass over the positions, instead of the
// FP64 tier's full recomputation.
__device__ bool overlap_exact(Smem &sm, const Ctx &c, int k)
{
    const int tid = threadIdx.x;
    const int i = c.k0 + k;
    const float4 a = sm.trial[k];
    const float4 *buf = stage_buf(sm);
    const double sig2 = c.ch->sig2;
    const float pre = (float)sig2 * (1.0f + 0x1p-12f);
    if (tid == 0) sm.ovl_flag = 0;
    for (int j0 = 0; j0 < c.N; j0 += GSTAGE) {
        stage_positions(sm, c, k, j0);
#pragma unroll 4
        for (int u = 0; u < GSTAGE / T; ++u) {
            const int t = u * T + tid, j = j0 + t;
            const float4 y = buf[t];
            const float dx = a.x - y.x, dy = a.y - y.y, dz = a.z - y.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2 < pre && j < c.N && j != i && d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < sig2) sm.ovl_flag = 1;
        }
    }
    bar_main();
    const bool o = sm.ovl_flag != 0;
    bar_main();
    return o;
}

__device__ __forceinline__ float4 pad_point(float v)
{
    return make_float4(v, v, v, 0.0f);
}

// Decision of move k from an interval [x_lo, x_hi] of its pair sum
// sum_j q_j (1/r' - 1/r).  Returns OUT_ACCEPT / OUT_METROPOLIS or -1.
__device__ __forceinline__ int decide_interval(const Smem &sm, int k, float lq, float x_lo, float x_hi)
{
    const float e1 = lq * x_lo, e2 = lq * x_hi;
    if (!(isfinite(e1) && isfinite(e2))) return -1;
    const float elo = fminf(e1, e2), ehi = fmaxf(e1, e2);
    const float L = sm.Lf[k];
    const float band = sm.bnd[k] + 0x1p-20f * (fmaxf(fabsf(elo), fabsf(ehi)) + fabsf(L));
    if (ehi < L - band) return OUT_ACCEPT;
    if (elo > L + band) return OUT_METROPOLIS;
    return -1;
}

// Overlap status of move k from the bits of its group's earlier ions: decided
// ions at their known position, undecided ions either way.
__device__ __forceinline__ void ingroup_overlap(const Smem &sm, int k, const unsigned *dec, const unsigned *acc,
                                                bool &certain, bool &possible)
{
    unsigned c = 0, p = 0;
#pragma unroll
    for (int w = 0; w < WORDS; ++w) {
        const unsigned bl = below(k, w);
        const unsigned dw = dec[w] & bl, uw = ~dec[w] & bl, aw = acc[w];
        c |= ((sm.ovn[k][w] & aw) | (sm.ovo[k][w] & ~aw)) & dw;
        c |= sm.ovo[k][w] & sm.ovn[k][w] & uw;
        p |= (sm.ovo[k][w] | sm.ovn[k][w]) & uw;
    }
    certain = c != 0;
    possible = p != 0;
}

// Partial sums of the decision rounds, two threads per move (half h of the
// earlier moves j in [64h, 64h + 64)): corrections of ions accepted since the
// last round (exact) and min/max sums over undecided ions (interval).  Uses
// the snapshot words acc0/dec0 and the words seen by the last round.
__device__ __forceinline__ void partial_pass(Smem &sm)
{
    const int tid = threadIdx.x;
    const int k = tid & (S - 1), h = tid >> 7;
    float sx = 0.f, lo = 0.f, hi = 0.f;
    if (!bit(sm.dec0, k)) {
        const int w0 = 2 * h, w1 = 2 * h + 1;
        const unsigned na0 = sm.acc0[w0] & ~sm.seen[w0] & below(k, w0), na1 = sm.acc0[w1] & ~sm.seen[w1] & below(k, w1);
        const unsigned un0 = ~sm.dec0[w0] & below(k, w0), un1 = ~sm.dec0[w1] & below(k, w1);
        if (na0 | na1 | un0 | un1) {
            const float *col = &sm.cin[(h * HALF) * CS + k];
#pragma unroll
            for (int jj = 0; jj < HALF; ++jj) {
                const unsigned na = jj < 32 ? na0 : na1, un = jj < 32 ? un0 : un1;
                const unsigned bm = 1u << (jj & 31);
                const float cv = col[jj * CS];
                sx += (na & bm) ? cv : 0.f;
                lo += (un & bm) ? fminf(cv, 0.f) : 0.f;
                hi += (un & bm) ? fmaxf(cv, 0.f) : 0.f;
            }
        }
    }
    sm.part[h][k] = sx;
    sm.plo[h][k] = lo;
    sm.phi[h][k] = hi;
    bar_main();
}

// ---------------------------------------------------------------------------
// Delayed acceptance, stage 1 (whole CTA), before the pair sums.  The in-group
// and window correction matrices are free until step 2a and hold the scratch.

// The reference (FP64) surrogate energy change of move k, identical to the oracle's arithmetic: near-field
// sums in ascending j, exact features, FP64 MLP with the series exp.  Whole CTA; uses the window matrix as
// scratch (free whenever this runs).  Returns the value in every thread.
__device__ double da_dEt64(Smem &sm, const Ctx &c, int k)
{
    const DADev &d = *c.ch->da;
    const int tid = threadIdx.x;
    const int Wg = min(d.W, c.B - 1);
    const int i = c.k0 + k;
    char *base = reinterpret_cast<char *>(sm.cwin);
    constexpr int LMAX = 1024;  // near-field terms per point (r_c <= 5 sigma: at most ~740 ions at contact density)
    double *sorted = reinterpret_cast<double *>(base);      // 2 x LMAX terms in ascending j (16384 B)
    int *F = reinterpret_cast<int *>(base + 16384);         // 2 x DA_FRS ints
    int *nl = reinterpret_cast<int *>(base + 16896);        // 2 counters
    int *lj = reinterpret_cast<int *>(base + 17024);        // 2 x LMAX indices (8192 B)
    double *lt = reinterpret_cast<double *>(base + 25216);  // 2 x LMAX terms (16384 B)
    double *hb = reinterpret_cast<double *>(base + 41600);  // 2 x 64 (h1) + 2 x 64 (h2)
    double *res = hb + 4 * DA_H;                            // phi0, phi1, g0, g1
    static_assert(41600 + 8 * (4 * DA_H + 8) <= S * CS * 4, "reference-surrogate scratch fits the window matrix");
    static_assert(2 * LMAX * 8 <= 16384 && 2 * DA_FRS * 4 <= 512, "scratch layout");
    const float4 x = sm.own[k], a = sm.trial[k];
    if (tid < 2 * DA_FRS) F[tid] = 0;
    if (tid < 2) nl[tid] = 0;
    bar_main();
    // near field and taper-region shells: counted candidates of the stencil cells, FP64 distances
    {
        const int G = d.nf_G;
        const int cx = da_ncell_axis(d, x.x), cy = da_ncell_axis(d, x.y), cz = da_ncell_axis(d, x.z);
        for (int cc = 0; cc < NF_ST; ++cc) {
            const int ax = cx + cc / 25 - 2, ay = cy + (cc / 5) % 5 - 2, az = cz + cc % 5 - 2;
            if (ax < 0 || ay < 0 || az < 0 || ax >= G || ay >= G || az >= G) continue;
            const int q = (ax * G + ay) * G + az;
            const int lo = __ldg(&d.cell_start[q]), hi = __ldg(&d.cell_start[q + 1]);
            for (int idx = lo + tid; idx < hi; idx += T) {
                const int j = __ldg(&d.cell_ions[idx]);
                if (!da_counted(i, c.g, c.B, Wg, j)) continue;
                const float4 y = __ldcg(&d.cell_pos[idx]);
#pragma unroll
                for (int pt = 0; pt < 2; ++pt) {
                    const float4 p = pt ? a : x;
                    const double dd2 = d2_fp64(p.x, p.y, p.z, y.x, y.y, y.z);
                    if (!(dd2 < d.rc2)) continue;
                    const int s = atomicAdd(&nl[pt], 1);
                    if (s < LMAX) {
                        lj[pt * LMAX + s] = j;
                        lt[pt * LMAX + s] = da_term64(d, (double)y.w, dd2);
                    }
                    if (dd2 >= d.rs2) {
                        const int kk = (int)floor(__dmul_rn(__ddiv_rn(__dsub_rn(dd2, d.rs2), __dsub_rn(d.rc2, d.rs2)), 32.0));
                        atomicAdd(&F[pt * DA_FRS + min(kk, 31)], (int)y.w);
                    }
                }
            }
        }
    }
    bar_main();
    // ascending-j order: each entry's rank among its list, then sequential sums
    for (int e = tid; e < 2 * LMAX; e += T) {
        const int pt = e / LMAX, s = e - pt * LMAX;
        const int n = min(nl[pt], LMAX);
        if (s < n) {
            const int jj = lj[pt * LMAX + s];
            int rank = 0;
            for (int u = 0; u < n; ++u) rank += lj[pt * LMAX + u] < jj;
            sorted[pt * LMAX + rank] = lt[pt * LMAX + s];
        }
    }
    bar_main();
    if (tid < 2) {
        double ph = 0.0;
        const int n = min(nl[tid], LMAX);
        for (int s = 0; s < n; ++s) ph = __dadd_rn(ph, sorted[tid * LMAX + s]);
        res[tid] = ph;
    }
    // MLP in FP64: 64 threads per point and layer, dot products in index order after the bias
    const unsigned short *w = d.w;
    if (tid < 2 * DA_H) {
        const int pt = tid / DA_H, o = tid - pt * DA_H;
        const float4 p = pt ? a : x;
        double z = (double)bf16f(__ldg(&w[DA_OFF_B1 + o]));
        for (int q = 0; q < 32; ++q)
            z = __dadd_rn(z, __dmul_rn((double)bf16f(__ldg(&w[o * DA_NIN + q])), __dmul_rn((double)F[pt * DA_FRS + q], 0.25)));
        const double px = p.x, py = p.y, pz = p.z;
        const double rad = __ddiv_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz))), d.R);
        z = __dadd_rn(z, __dmul_rn((double)bf16f(__ldg(&w[o * DA_NIN + 32])), rad));
        hb[pt * DA_H + o] = silu64(z);
    }
    bar_main();
    if (tid < 2 * DA_H) {
        const int pt = tid / DA_H, o = tid - pt * DA_H;
        double z = (double)bf16f(__ldg(&w[DA_OFF_B2 + o]));
        for (int q = 0; q < DA_H; ++q)
            z = __dadd_rn(z, __dmul_rn((double)bf16f(__ldg(&w[DA_OFF_W2 + o * DA_H + q])), hb[pt * DA_H + q]));
        hb[2 * DA_H + pt * DA_H + o] = silu64(z);
    }
    bar_main();
    if (tid < 2) {
        double gg = (double)bf16f(__ldg(&w[DA_OFF_B3]));
        for (int q = 0; q < DA_H; ++q)
            gg = __dadd_rn(gg, __dmul_rn((double)bf16f(__ldg(&w[DA_OFF_W3 + q])), hb[2 * DA_H + tid * DA_H + q]));
        res[2 + tid] = gg;
    }
    bar_main();
    const double lq = __dmul_rn(c.ch->lB, (double)x.w);
    const double v = __dmul_rn(lq, __dsub_rn(__dadd_rn(res[1], res[3]), __dadd_rn(res[0], res[2])));
    bar_main();
    return v;
}

// Bounded wait until the ledger has folded every group up to `need` (stream index s * B + g).
__device__ bool wait_ledger(const ChainDev &ch, unsigned long long need, Ctl *ctl)
{
    unsigned long long t0 = 0;  // started at the first check
    unsigned spins = 0;
    while (ld_acquire(ch.ledger_seq) < need) {
        if (*(volatile int *)&ctl->abort) return false;
        if (++spins > 16) __nanosleep(64);
        if ((spins & 63) == 0) {
            const unsigned long long now = globaltimer();
            if (t0 == 0) t0 = now;
            else if ((long long)(now - t0) > ctl->timeout_ns) {
                atomicCAS(&ctl->err, 0, KERR_TIMEOUT);
                atomicExch(&ctl->abort, 1);
                return false;
            }
        }
    }
    return true;
}

// Stage 1 of delayed acceptance for the whole group (whole CTA).  Decides the moves it rejects (overlap
// with a counted ion, or the surrogate test), lists the survivors, and gives each survivor its stage-2
// threshold Lf = L(u2) + dEt with the surrogate's error added to dEtB.
__device__ bool da_stage1(Smem &sm, const Ctx &c, Ctl *ctl, int mode, int &n_fp64, long long *part)
{
    const ChainDev &ch = *c.ch;
    const DADev &d = *ch.da;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nk = c.nk, Wg = min(d.W, c.B - 1);
    const float lBf = (float)ch.lB;
    if (tid == 0) {
        const unsigned long long need = c.s * (unsigned long long)c.B + (unsigned long long)max(c.g - Wg, 0);
        sm.ok = wait_ledger(ch, need, ctl) ? 1 : 0;
    }
    bar_main();
    if (!sm.ok) return false;
    char *base = reinterpret_cast<char *>(sm.cin);
    float *Wf = reinterpret_cast<float *>(base);                // DA_NP floats
    int *Fr = reinterpret_cast<int *>(base + 25616);            // 2S shell histograms (old positions, then trials)
    float *w2n = reinterpret_cast<float *>(base + 59408);
    float *gv = reinterpret_cast<float *>(base + 59664);
    float *ge = gv + 2 * S;
    float *nph0 = ge + 2 * S, *nph1 = nph0 + S, *nA0 = nph1 + S, *nA1 = nA0 + S;
    int *nnt = reinterpret_cast<int *>(nA1 + S), *novl = nnt + S;
    int *wsc = novl + S;  // per warp: 256 ints of near-field stencil scratch
    static_assert(59664 + 4 * 2 * S * 2 + 4 * 4 * S + 4 * 2 * S + 4 * 256 * (T / 32) <= 2 * S * CS * 4, "stage-1 scratch");
    for (int q = tid; q < DA_NP; q += T) Wf[q] = bf16f(__ldg(&d.w[q]));
    if (tid < DA_H) w2n[tid] = __ldg(&d.w2n[tid]);
    for (int q = tid; q < 2 * S * DA_FRS; q += T) Fr[q] = 0;
    if (tid < WORDS) sm.d64w[tid] = 0u;
    if (tid == 0) sm.namb = 0;
    bar_main();
    const auto active = [&](int k) { return k < nk && !(sm.st[k] & (ST_INACTIVE | ST_WALL)); };
    // near field and taper-region shell histograms (warp per move)
    long long tq = clock64();
    for (int k = warp; k < nk; k += T / 32) {
        if (!active(k)) continue;
        const NearOut o = da_near_warp(d, c.g, c.B, Wg, c.k0 + k, sm.own[k], sm.trial[k], ch.sig2_lo, ch.sig2_hi, ch.sig2,
                                       Fr + k * DA_FRS, Fr + (S + k) * DA_FRS, wsc + 256 * warp);
        if (lane == 0) {
            nph0[k] = o.ph0;
            nph1[k] = o.ph1;
            nA0[k] = o.A0;
            nA1[k] = o.A1;
            nnt[k] = o.nt;
            novl[k] = o.ovl;
        }
    }
    bar_main();
    part[3] += clock64() - tq;
    tq = clock64();
    // MLP at every point (thread = point: 0..S-1 old positions, S..2S-1 trials); with all weights zero g = 0
    // exactly (every layer's output is silu(0) = 0 and the last one is 0), so the pass is skipped
    {
        const int k = tid & (S - 1);
        float g = 0.f, eg = 0.f;
        if (active(k) && !novl[k] && !d.mlp_zero) {
            const float4 p = tid < S ? sm.own[k] : sm.trial[k];
            float v[DA_NIN];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = (float)Fr[tid * DA_FRS + q] * 0.25f;
            v[32] = da_radial32(d, p);
            da_mlp32(Wf, w2n, v, g, eg);
        }
        gv[tid] = g;
        ge[tid] = eg;
    }
    bar_main();
    part[2] += clock64() - tq;
    // FP32 surrogate energy change and its bound; stage-1 decisions outside the band
    if (tid < S) {
        const int k = tid;
        unsigned stv = sm.st[k];
        sm.dEt32[k] = __int_as_float(0x7fc00000);
        sm.dEtB[k] = 0.f;
        sm.dEt64[k] = __longlong_as_double(0x7ff8000000000000ll);
        if (active(k)) {
            if (novl[k]) {
                sm.outcome[k] = (signed char)OUT_OVERLAP;
                sm.tier[k] = 6;
                stv |= ST_DA_DONE;
            } else {
                const float lq = lBf * sm.own[k].w;
                const float ph0 = nph0[k], ph1 = nph1[k], g0 = gv[k], g1 = gv[S + k];
                const float cph = ((float)nnt[k] + 40.0f) * U32;  // per term <= 34u of |q|/d (taper included)
                const float dEt = lq * ((ph1 + g1) - (ph0 + g0));
                const float E = fabsf(lq) *
                                    (cph * (nA0[k] + nA1[k]) + ge[k] + ge[S + k] +
                                     3.0f * U32 * (fabsf(ph1) + fabsf(g1) + fabsf(ph0) + fabsf(g0))) *
                                    (1.0f + 0x1p-10f) +
                                3.0f * U32 * fabsf(dEt);
                sm.dEt32[k] = dEt;
                sm.dEtB[k] = E;
                int dec = 1;
                if (!(stv & ST_UZERO)) {
                    const float L = sm.Lf[k];
                    const float b = (mode == 1 || mode == 3) ? finf()
                                                             : (mode == 2 ? 0.f : E + 0x1p-20f * (fabsf(dEt) + fabsf(L)));
                    dec = (dEt < L - b) ? 1 : ((dEt > L + b) ? 0 : -1);
                }
                if (dec == 0) {
                    sm.outcome[k] = (signed char)OUT_DA1;
                    sm.tier[k] = 6;
                    stv |= ST_DA_DONE;
                } else if (dec < 0) {
                    sm.damb[atomicAdd(&sm.namb, 1)] = k;
                }
            }
            sm.st[k] = (unsigned char)stv;
        }
    }
    bar_main();
    // stage-1 decisions inside the band: the reference arithmetic
    const int na = sm.namb;
    for (int e = 0; e < na; ++e) {
        const int k = sm.damb[e];
        const double v = da_dEt64(sm, c, k);
        if (tid == 0) {
            sm.dEt64[k] = v;
            sm.d64w[k >> 5] |= 1u << (k & 31);
            const unsigned long long m = c.s * (unsigned long long)c.N + (unsigned long long)(c.k0 + k);
            const unsigned u1 = move_draws(ch, m, 0u).w >> 8;
            const bool pass = (u1 == 0u) || v < -series_log((double)u1 * 0x1p-24);
            if (!pass) {
                sm.outcome[k] = (signed char)OUT_DA1;
                sm.tier[k] = 7;
                sm.st[k] = (unsigned char)(sm.st[k] | ST_DA_DONE);
            }
        }
        bar_main();
    }
    n_fp64 += na;
    // survivors in ascending order, and their stage-2 thresholds
    if (tid < S) {
        const int k = tid;
        const bool sv = active(k) && !(sm.st[k] & ST_DA_DONE);
        const unsigned bal = __ballot_sync(FULL, sv);
        if (lane == 0) sm.redf[warp] = __int_as_float(__popc(bal));
        if (sv) {
            const unsigned long long m = c.s * (unsigned long long)c.N + (unsigned long long)(c.k0 + k);
            const unsigned u2 = move_draws(ch, m, 1u).w >> 8;
            unsigned stv = sm.st[k] & ~ST_UZERO;
            const bool exact = bit(sm.d64w, k);
            const float dEt = exact ? (float)sm.dEt64[k] : sm.dEt32[k];
            const float E = exact ? 2.0f * U32 * fabsf(dEt) : sm.dEtB[k];
            float L2 = finf();
            if (u2 == 0u) stv |= ST_UZERO;
            else L2 = -logf(__uint2float_rn(u2) * 0x1p-24f);
            const float Lf = L2 + dEt;
            sm.Lf[k] = Lf;
            sm.dEtB[k] = (u2 == 0u) ? 0.f : (E + 0x1p-20f * (fabsf(L2) + fabsf(dEt)) + 2.0f * U32 * fabsf(Lf)) * (1.0f + 0x1p-10f);
            sm.st[k] = (unsigned char)stv;
        }
    }
    bar_main();
    if (tid < S) {
        const int k = tid, w = k >> 5;
        int before = 0;
        for (int q = 0; q < w; ++q) before += __float_as_int(sm.redf[q]);
        const bool sv = active(k) && !(sm.st[k] & ST_DA_DONE);
        const unsigned bal = __ballot_sync(FULL, sv);
        const int n = before + __popc(bal & ((1u << lane) - 1u));
        if (sv) sm.surv[n] = (unsigned char)k;
        sm.slot[k] = sv ? (unsigned char)n : (unsigned char)255;
        if (k == S - 1) sm.ns = before + __popc(bal);
    }
    bar_main();
    return true;
}

// Stage 1 of the overlap prefilter (a chain without a surrogate whose DADev is a prefilter): the moves whose trial
// overlaps a counted ion are rejected as overlaps (the reference chain rejects them too, whatever their energy
// change), the others are listed as survivors and decided by the plain chain's rule on their exact dE: the
// acceptance draw, threshold and band of step 1 are left as they are.
__device__ bool prefilter_stage1(Smem &sm, const Ctx &c, Ctl *ctl)
{
    const ChainDev &ch = *c.ch;
    const DADev &d = *ch.da;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nk = c.nk, Wg = min(d.W, c.B - 1);
    if (tid == 0) {
        const unsigned long long need = c.s * (unsigned long long)c.B + (unsigned long long)max(c.g - Wg, 0);
        sm.ok = wait_ledger(ch, need, ctl) ? 1 : 0;
        sm.namb = 0;
    }
    if (tid < WORDS) sm.d64w[tid] = 0u;
    if (tid < S) {
        sm.dEt32[tid] = __int_as_float(0x7fc00000);
        sm.dEtB[tid] = 0.f;
        sm.dEt64[tid] = __longlong_as_double(0x7ff8000000000000ll);
    }
    bar_main();
    if (!sm.ok) return false;
    const auto active = [&](int k) { return k < nk && !(sm.st[k] & (ST_INACTIVE | ST_WALL)); };
    for (int k = warp; k < nk; k += T / 32) {  // warp per move
        if (!active(k)) continue;
        const int o = da_ovl_warp(d, c.g, c.B, Wg, c.k0 + k, sm.own[k], sm.trial[k], ch.sig2_lo, ch.sig2_hi, ch.sig2);
        if (lane == 0 && o) {
            sm.outcome[k] = (signed char)OUT_OVERLAP;
            sm.tier[k] = 6;
            sm.st[k] = (unsigned char)(sm.st[k] | ST_DA_DONE);
        }
    }
    bar_main();
    bool sv = false;
    if (tid < S) {
        sv = active(tid) && !(sm.st[tid] & ST_DA_DONE);
        const unsigned bal = __ballot_sync(FULL, sv);
        if (lane == 0) sm.redf[warp] = __int_as_float(__popc(bal));
    }
    bar_main();
    if (tid < S) {
        const int k = tid, w = k >> 5;
        int before = 0;
        for (int q = 0; q < w; ++q) before += __float_as_int(sm.redf[q]);
        const unsigned bal = __ballot_sync(FULL, sv);
        const int n = before + __popc(bal & ((1u << lane) - 1u));
        if (sv) sm.surv[n] = (unsigned char)k;
        sm.slot[k] = sv ? (unsigned char)n : (unsigned char)255;
        if (k == S - 1) sm.ns = before + __popc(bal);
    }
    bar_main();
    return true;
}

// One work item: the S moves of group g of chain `tk.chain` at sweep s.
// role 0: the whole work item (the cluster's leader in pairs mode: even tiles); role 1: the pairs-mode helper,
// which sums the odd tiles for the leader and decides nothing.
// Groups staged in the buffer after the one holding groups up to in - 1: the consecutive groups in, in + 1, ... that
// exist (< ntl) and lie inside the publication horizon hz, at most TG; 0 when group in is not known to be published.
__device__ __forceinline__ int next_groups(int in, int ntl, int hz)
{
    int pn = 0;
#pragma unroll
    for (int k = 0; k < TG; ++k)
        if (pn == k && in + k < ntl && in + k <= hz) pn = k + 1;
    return pn;
}

// One buffer of the tile ring against the thread's moves: cnt staged groups of S ions, column slices of NSL (8 for
// one group of warps, 16 when the helper warps take slices 8..15), this thread's slice r0.  Only the occupied
// 32-move layers run (nm of them): one packed pair for <= 2, a packed pair and the third layer alone for 3, two
// packed pairs for 4; an empty slot in the last layer repeats a real move and is never written back.  The FP32
// partial sums s2 are promoted into the float-float sums (hA, lA) after every group, so no partial sum holds more
// than S / NSL <= 16 terms (the band's C_SUM).
template <int NSL>
__device__ __forceinline__ void tile_buffer(const float4 *tile, int cnt, int r0, int nm, const Mv2 (&mv)[MPT / 2],
                                            f32x2 (&s2)[MPT / 2], f32x2 (&P2)[MPT / 2], float (&mA)[MPT],
                                            float (&hA)[MPT], float (&lA)[MPT])
{
    constexpr int NJ = S / NSL;  // partners per thread per group
    for (int gq = 0; gq < cnt; ++gq) {
        const float4 *tg = tile + gq * S + r0;
        if (nm <= 2) {
#pragma unroll 4
            for (int jj = 0; jj < NJ; ++jj) pair_far2(mv[0], tg[jj * NSL], s2[0], P2[0], mA[0], mA[1]);
        } else if (nm == 3) {
            float s3, s3b, p3, p3b;
            upk2(s2[1], s3, s3b);
            upk2(P2[1], p3, p3b);
#pragma unroll 4
            for (int jj = 0; jj < NJ; ++jj) {
                const float4 y = tg[jj * NSL];
                pair_far2(mv[0], y, s2[0], P2[0], mA[0], mA[1]);
                pair_far1(mv[1], y, s3, p3, mA[2]);
            }
            s2[1] = pk2(s3, s3b);
            P2[1] = pk2(p3, p3b);
        } else {
#pragma unroll 4
            for (int jj = 0; jj < NJ; ++jj) {
                const float4 y = tg[jj * NSL];
                pair_far2(mv[0], y, s2[0], P2[0], mA[0], mA[1]);
                pair_far2(mv[1], y, s2[1], P2[1], mA[2], mA[3]);
            }
        }
#pragma unroll
        for (int pp = 0; pp < MPT / 2; ++pp) {  // promote this group's partial sums
            float v[2];
            upk2(s2[pp], v[0], v[1]);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                float t2, e;
                two_sum(hA[2 * pp + u], v[u], t2, e);
                hA[2 * pp + u] = t2;
                lA[2 * pp + u] += e;
            }
            s2[pp] = pk2(0.f, 0.f);
        }
    }
}

// One buffer for a group of 65..72 occupied move slots ("excess" mode): the first 64 slots as two
// layers (mv0: slots p and p + 32 of thread row p, column slices of SL, as tile_buffer), and the e = ns - 64
// excess moves by rows of XR = T / XS threads, XS column slices each: row q < e runs excess move 64 + q (mx, lane 0)
// against ions rx, rx + XS, ... of each group.  The excess sums are promoted after every group like the others
// (S / XS <= 16 terms per partial sum) and handed over through shared memory after the tiles.
template <int XS>
__device__ __forceinline__ void tile_buffer_x(const float4 *tile, int cnt, int r0, const Mv2 &mv0, f32x2 &s20,
                                              f32x2 &P20, float &mA0, float &mA1, float &hA0, float &lA0, float &hA1,
                                              float &lA1, bool xact, int rx, const Mv2 &mx, float &sx, float &Px,
                                              float &mnx, float &hx, float &lx)
{
    constexpr int NJ = S / SL, NX = S / XS;
    for (int gq = 0; gq < cnt; ++gq) {
        const float4 *tg = tile + gq * S;
#pragma unroll 4
        for (int jj = 0; jj < NJ; ++jj) pair_far2(mv0, tg[r0 + jj * SL], s20, P20, mA0, mA1);
        if (xact) {
#pragma unroll
            for (int jj = 0; jj < NX; ++jj) pair_far1(mx, tg[rx + jj * XS], sx, Px, mnx);
            float t2, e;
            two_sum(hx, sx, t2, e);
            hx = t2;
            lx += e;
            sx = 0.f;
        }
        float v0, v1, t2, e;
        upk2(s20, v0, v1);
        two_sum(hA0, v0, t2, e);
        hA0 = t2;
        lA0 += e;
        two_sum(hA1, v1, t2, e);
        hA1 = t2;
        lA1 += e;
        s20 = pk2(0.f, 0.f);
    }
}

// The packed move data of thread row p (move slots p + 32 m) from the staged positions: old positions, the
// displacements and their negatives.
__device__ __forceinline__ void tile_moves(const Smem &sm, int p, int ns, int (&km)[MPT], Mv2 (&mv)[MPT / 2])
{
    float3 b3[MPT], d3[MPT];
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        km[m] = (p + 32 * m < ns) ? (int)sm.surv[p + 32 * m] : -1;
        const int kk = km[m] < 0 ? 0 : km[m];
        const float4 a = sm.trial[kk], b = sm.own[kk];
        b3[m] = make_float3(b.x, b.y, b.z);
        d3[m] = make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
    }
#pragma unroll
    for (int pp = 0; pp < MPT / 2; ++pp) mv[pp] = make_mv2(b3[2 * pp], d3[2 * pp], b3[2 * pp + 1], d3[2 * pp + 1]);
}

// The helper warps (threads T..2T-1 of the 2T-thread kernel): column slices 8..15 of every work item's tile pass,
// in step with the work-item warps at barrier 2.  Per item: the hand-over barrier (command RUN, SKIP or EXIT, and
// the tile count, in the slot of the hand-over's parity: the work-item warps write the other slot next, so a slow
// helper never reads a newer command), the tile loop with the same barriers and the same decisions as the
// work-item warps (all read from shared memory written before the barrier that precedes the read), then the
// per-move sums into shared memory and the closing barrier.  After an abort seen in the loop both sides leave the
// item; the work-item warps then send EXIT.
__device__ void helper_loop(Smem &sm)
{
    const int ht = threadIdx.x - T;
    const int p = ht / SL, r = ht % SL;
    int hseq = 0;
    for (;;) {
        bar_all();  // hand-over
        const int cmd = sm.hcmd[hseq & 1], ntl = sm.hntl[hseq & 1];
        ++hseq;
        if (cmd == HC_EXIT) return;
        if (cmd != HC_RUN) continue;
        const int ns = sm.ns, nm = (ns + 31) / 32;
        int km[MPT];
        Mv2 mv[MPT / 2];
        tile_moves(sm, p, ns, km, mv);
        f32x2 s2[MPT / 2], P2[MPT / 2];
        float hA[MPT], lA[MPT], mA[MPT];
#pragma unroll
        for (int pp = 0; pp < MPT / 2; ++pp) {
            s2[pp] = pk2(0.f, 0.f);
            P2[pp] = pk2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            hA[m] = lA[m] = 0.f;
            mA[m] = finf();
        }
        bool ok = true;
        int it = 0;
        for (int i = 0; i < ntl; ++it) {
            const int cur = it & 1;
            const int cnt = sm.tcnt[cur];
            const int hz = sm.hzs[cur];
            const int in = i + cnt;
            const int pn = next_groups(in, ntl, hz);
            tile_buffer<2 * SL>(sm.tile[cur], cnt, SL + r, nm, mv, s2, P2, mA, hA, lA);
            bar_all();  // the iteration's barrier
            if (in < ntl && pn == 0) {
                bar_all();  // the next tile has been waited for
                if (!sm.ok) {
                    ok = false;
                    break;
                }
                bar_all();  // ... and staged
            }
            i = in;
        }
        if (!ok) continue;
        float PA[MPT];
#pragma unroll
        for (int pp = 0; pp < MPT / 2; ++pp) upk2(P2[pp], PA[2 * pp], PA[2 * pp + 1]);
#pragma unroll
        for (int o = 1; o < SL; o <<= 1) {
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                const float h2 = __shfl_xor_sync(FULL, hA[m], o), l2 = __shfl_xor_sync(FULL, lA[m], o);
                float t2, e;
                two_sum(hA[m], h2, t2, e);
                hA[m] = t2;
                lA[m] = lA[m] + l2 + e;
                PA[m] += __shfl_xor_sync(FULL, PA[m], o);
                mA[m] = fminf(mA[m], __shfl_xor_sync(FULL, mA[m], o));
            }
        }
        if (r < MPT) {  // lane r of each slice group stores move slot m = r
#pragma unroll
            for (int m = 0; m < MPT; ++m)
                if (r == m && km[m] >= 0) {
                    help_h(sm)[km[m]] = hA[m];
                    help_l(sm)[km[m]] = lA[m];
                    help_p(sm)[km[m]] = PA[m];
                    help_m(sm)[km[m]] = mA[m];
                }
        }
        bar_all();  // the sums are in shared memory
    }
}

template <bool HELP, bool DA>
__device__ bool process_group(Smem &sm, const ChainDev *__restrict__ chains, const Ticket tk, int ticket, Ctl *ctl,
                              int role, int &hseq)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const bool pairs = ctl->pairs != 0, helper = role == 1;
    // the shared guard: in the instance for chains with a cell list only (on the plain instance the board's code
    // measured slower, through the register allocation of the tile loop)
    constexpr bool SHG = DA && !HELP;
    const ChainDev &ch = chains[tk.chain];
    Ctx c;
    c.ch = &ch;
    c.N = ch.N;
    c.B = ch.B;
    c.g = tk.g;
    c.k0 = c.g * S;
    c.nk = min(S, c.N - c.k0);
    c.s = *ch.sweep + (unsigned long long)tk.s_rel;
    const unsigned long long s = c.s;
    c.Pprev = ch.pos[s & 1];
    c.Pcur = ch.pos[(s + 1) & 1];
    const int N = c.N, B = c.B, g = c.g, k0 = c.k0, nk = c.nk;
    const unsigned tag_prev = (unsigned)s, tag_cur = (unsigned)(s + 1);
    // the window: the group moved just before this one, when it exists in this run of the chain
    unsigned long long sw = 0;
    c.Jw = -1;
    c.win = false;
    c.nwk = 0;
    if (B >= 2) {
        c.Jw = (g == 0) ? B - 1 : g - 1;
        sw = (g == 0) ? s - 1 : s;
        c.win = (g == 0) ? (s > ch.sweep_base) : true;
        c.nwk = min(S, N - c.Jw * S);
    }
    // deep windows: the groups g-2, g-3, ... before the window that belong to this sweep (always full groups);
    // unless disabled (MC_OPT_DEEP_WINDOWS), otherwise those groups are ordinary tiles
    c.nd = (c.win && ctl->deep) ? max(0, min(DW, g - 1)) : 0;
    const float lo2 = ch.sig2_lo, hi2 = ch.sig2_hi;
    const double sig2 = ch.sig2;
    const float s2f = (float)sig2;
    const float sp = sqrtf(s2f) * (1.0f - 0x1p-17f);  // settled ions of a valid move are at least this far
    const int mode = ctl->guard_mode;
    const float lBf = (float)ch.lB;
    // phase timers (thread 0): SM cycles
    long long cyc_start = clock64(), cyc_tiles = 0, cyc_win = 0, cyc_guard = 0, cyc_res0 = 0, cyc_ovl = 0;
    int n_scan = 0;
    long long cyc_t[3] = {0, 0, 0};
    const bool trc = ch.trace != nullptr;  // timeline stamps only while a trace is recorded
    const unsigned long long gt_start = trc ? globaltimer() : 0ull;
    unsigned long long gt_ready = 0, gt_window = 0, gt_resolved = 0, gt_pub = 0, gt_tile = 0, gt_tiles = 0, gt_w2 = 0;
    unsigned long long gt_ph[4] = {0, 0, 0, 0};
    long long cw0 = 0;
    unsigned cres[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned tbase = sm.tmem + ((unsigned)(32 * (warp & 3)) << 16);  // this warp's TMEM lane quarter
    int n_rounds = 0;

    // 1. own positions (version s-1) and, if active, the window's old positions (version sw-1)
    if (warp == 0) {
        unsigned bits;
        bool ok = wait_words(ch, g, (nk + 31) / 32, tag_prev, tag_prev, ctl, bits, true, false, SHG);
        if (ok && c.win) ok = wait_words(ch, c.Jw, (c.nwk + 31) / 32, (unsigned)sw, (unsigned)(sw + 1), ctl, bits, true, false, SHG);
        for (int d = 0; ok && d < c.nd; ++d)  // deep windows: version s-1 (their version s may be out already)
            ok = wait_words(ch, g - 2 - d, WORDS, tag_prev, tag_cur, ctl, bits, true, false, SHG);
        if (lane == 0) sm.ok = ok;
    }
    bar_main();
    if (!sm.ok) return false;
    if (tid < S) {
        const int k = tid;
        unsigned stv = 0;
        if (k < nk) {
            const float4 x = __ldcg(&c.Pprev[k0 + k]);
            const unsigned long long m = s * (unsigned long long)N + (unsigned long long)(k0 + k);
            const uint4 w = move_draws(ch, m, 0u);
            const float4 a = make_float4(trial_coord(x.x, w.x, ch.D), trial_coord(x.y, w.y, ch.D),
                                         trial_coord(x.z, w.z, ch.D), x.w);
            sm.own[k] = x;
            sm.trial[k] = a;
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn((double)a.x, (double)a.x), __dmul_rn((double)a.y, (double)a.y)),
                                        __dmul_rn((double)a.z, (double)a.z));
            if (r2 > ch.Rc2) stv |= ST_WALL;
            const unsigned ua = w.w >> 8;
            if (ua == 0u) {
                stv |= ST_UZERO;
                sm.Lf[k] = finf();
            } else {
                sm.Lf[k] = -logf(__uint2float_rn(ua) * 0x1p-24f);
            }
        } else {
            sm.own[k] = pad_point(-1.0e6f);
            sm.trial[k] = pad_point(-1.0e6f);
            sm.Lf[k] = 0.f;
            stv = ST_INACTIVE;
        }
        if (c.win && k < c.nwk) {
            const int jg = c.Jw * S + k;
            const float4 x = __ldcg(&ch.pos[sw & 1][jg]);
            const unsigned long long m = sw * (unsigned long long)N + (unsigned long long)jg;
            const uint4 w = move_draws(ch, m, 0u);
            sm.wold[k] = x;
            sm.wtri[k] = make_float4(trial_coord(x.x, w.x, ch.D), trial_coord(x.y, w.y, ch.D),
                                     trial_coord(x.z, w.z, ch.D), x.w);
        }
        for (int d = 0; d < c.nd; ++d) {
            const int jg = (g - 2 - d) * S + k;
            const float4 x = __ldcg(&c.Pprev[jg]);
            const uint4 w = move_draws(ch, s * (unsigned long long)N + (unsigned long long)jg, 0u);
            sm.dold[d][k] = x;
            sm.dtri[d][k] = make_float4(trial_coord(x.x, w.x, ch.D), trial_coord(x.y, w.y, ch.D),
                                        trial_coord(x.z, w.z, ch.D), x.w);
        }
        sm.wexd[k] = 0.f;
        sm.st[k] = (unsigned char)stv;
        sm.outcome[k] = -1;
        sm.tier[k] = 0;
        sm.dEv[k] = 0.0;
#pragma unroll
        for (int w = 0; w < WORDS; ++w) {
            sm.ovo[k][w] = 0u;
            sm.ovn[k][w] = 0u;
            sm.wovo[k][w] = 0u;
            sm.wovn[k][w] = 0u;
#pragma unroll
            for (int d = 0; d < DW; ++d) {
                sm.dovo[d][k][w] = 0u;
                sm.dovn[d][k][w] = 0u;
            }
        }
    }
    if (tid < WORDS) {
        sm.accw[tid] = 0u;
        sm.decw[tid] = 0u;
        sm.seen[tid] = 0u;
        sm.winacc[tid] = 0u;
#pragma unroll
        for (int d = 0; d < DW; ++d) sm.dacc[d][tid] = 0u;
    }
    bar_main();

    // 1b. delayed acceptance: stage 1 decides what it can before any pair sum; only survivors continue
    int n_dfp64 = 0;
    long long da_part[4] = {0, 0, 0, 0};
    const long long cyc_da0 = clock64();
    if (DA && ch.da) {
        if (!(ch.pf ? prefilter_stage1(sm, c, ctl) : da_stage1(sm, c, ctl, mode, n_dfp64, da_part))) return false;
    } else {
        if (tid < S) {
            sm.surv[tid] = (unsigned char)tid;
            sm.slot[tid] = tid < nk ? (unsigned char)tid : (unsigned char)255;
        }
        if (tid == 0) sm.ns = nk;
        bar_main();
    }
    const long long cyc_da = clock64() - cyc_da0;
    const int ns = sm.ns;
    const int nm = (ns + 31) / 32;  // occupied layers of 32 move slots

    // 2. pair sums.  Thread (p, r): moves p + 32 m (m = 0..3), column slice r of 8.
    const int p = tid / SL, r = tid % SL;
    float4 a[MPT], b[MPT];
    float3 b3[MPT], d3[MPT];
    float sA[MPT], hA[MPT], lA[MPT], AA[MPT], TA[MPT], CA[MPT], PA[MPT], mA[MPT];
    int km[MPT];  // the move in each slot (-1: empty)
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        km[m] = (p + 32 * m < ns) ? (int)sm.surv[p + 32 * m] : -1;
        const int kk = km[m] < 0 ? 0 : km[m];
        a[m] = sm.trial[kk];
        b[m] = sm.own[kk];
        b3[m] = make_float3(b[m].x, b[m].y, b[m].z);
        d3[m] = make_float3(a[m].x - b[m].x, a[m].y - b[m].y, a[m].z - b[m].z);
        sA[m] = hA[m] = lA[m] = AA[m] = TA[m] = CA[m] = PA[m] = 0.f;
        mA[m] = finf();
    }
    auto promote = [&]() {
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            float s2, e;
            two_sum(hA[m], sA[m], s2, e);
            hA[m] = s2;
            lA[m] += e;
            sA[m] = 0.f;
        }
    };

    if (!helper) {  // the helper sums tiles only
    // 2a. this group: upper triangle final (Algorithm 3), lower triangle both ways (Algorithm 4)
    for (int j = r; j < nk; j += SL) {
        const float4 yo = sm.own[j], yn = sm.trial[j];
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int k = km[m];
            if (k < 0 || j == k) continue;
            if (j > k) pair_far(b3[m], d3[m], yo, sA[m], TA[m], PA[m], mA[m]);
            else both_pair(sm.cin, sm.ovo, sm.ovn, k, j, a[m], b[m], yo, yn, sA[m], AA[m], TA[m], CA[m], lo2, hi2, sig2);
        }
    }
    promote();
    // 2b. the window group, both ways
    if (c.win) {
        for (int j = r; j < c.nwk; j += SL) {
            const float4 yo = sm.wold[j], yn = sm.wtri[j];
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                const int k = km[m];
                if (k < 0) continue;
                both_pair(sm.cwin, sm.wovo, sm.wovn, k, j, a[m], b[m], yo, yn, sA[m], AA[m], TA[m], CA[m], lo2, hi2,
                          sig2);
            }
        }
        promote();
    }

    // 2b2. deep windows, both positions.  Warp (q, h): move slots 32 q + lane, ions [64 h, 64 h + 64) of each
    // deep window.  The corrections go to TMEM (lane = slot, column = S d + j) and are summed over the accepted
    // ions after the tiles, when the deep windows' bits are out (group-times before the window's); old-position
    // terms (float-float, 16 terms per FP32 partial) and bound sums per (half, slot) in shared memory, merged
    // in 2d.
    if (c.nd > 0) {
        const int q = warp & 3, h = warp >> 2, n = 32 * q + lane;
        const bool act = n < ns;
        const int k = act ? (int)sm.surv[n] : 0;
        float sh = 0.f, sl = 0.f, A = 0.f, Tt = 0.f, TC = 0.f, lo0 = 0.f, hi0 = 0.f;
        if (32 * q < ns) {  // warp-uniform: TMEM stores are whole-warp instructions
            const float4 ak = sm.trial[k], bk = sm.own[k];
            for (int d = 0; d < c.nd; ++d) {
                unsigned ow0 = 0u, ow1 = 0u, nw0 = 0u, nw1 = 0u;
#pragma unroll 1
                for (int q16 = 0; q16 < HALF / 16; ++q16) {
                    float v[16];
                    float p16 = 0.f;
                    unsigned o16 = 0u, n16 = 0u;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int j = h * HALF + 16 * q16 + i;
                        const float4 yo = sm.dold[d][j], yn = sm.dtri[d][j];
                        float Ao, An, d2o, d2n;
                        const float to = pair_term(ak, bk, yo, Ao, d2o);
                        const float tn = pair_term(ak, bk, yn, An, d2n);
                        const float cv = tn - to;
                        p16 += to;
                        Tt += fabsf(to);
                        A += Ao + An;
                        TC += fabsf(cv);
                        if (d == 0) {
                            lo0 += fminf(cv, 0.f);
                            hi0 += fmaxf(cv, 0.f);
                        }
                        v[i] = cv;
                        if (overlaps(d2o, ak, yo, lo2, hi2, sig2)) o16 |= 1u << i;
                        if (overlaps(d2n, ak, yn, lo2, hi2, sig2)) n16 |= 1u << i;
                    }
                    float s2, e;
                    two_sum(sh, p16, s2, e);
                    sh = s2;
                    sl += e;
                    const int sh16 = 16 * (q16 & 1);
                    if (q16 < 2) {
                        ow0 |= o16 << sh16;
                        nw0 |= n16 << sh16;
                    } else {
                        ow1 |= o16 << sh16;
                        nw1 |= n16 << sh16;
                    }
                    __syncwarp();
                    tmem_st16(tbase + (unsigned)(S * d + h * HALF + 16 * q16), v);
                }
                if (act) {
                    sm.dovo[d][k][2 * h] = ow0;
                    sm.dovo[d][k][2 * h + 1] = ow1;
                    sm.dovn[d][k][2 * h] = nw0;
                    sm.dovn[d][k][2 * h + 1] = nw1;
                }
            }
            // every store waited for itself; no whole-warp tcgen05 instruction follows the divergent branch above
        }
        sm.dsh[h][n] = act ? sh : 0.f;
        sm.dsl[h][n] = act ? sl : 0.f;
        sm.dsA[h][n] = act ? A : 0.f;
        sm.dsT[h][n] = act ? Tt : 0.f;
        sm.dsC[h][n] = act ? TC : 0.f;
        sm.dlo[h][n] = act ? lo0 : 0.f;
        sm.dhi[h][n] = act ? hi0 : 0.f;
    }

    // 2b'. interval sums of the corrections (threads < S: this group, threads >= S: the window);
    // needs only the two passes above, so it runs before the tiles
    bar_main();
    {
        const int k = tid & (S - 1), h = tid >> 7;
        float lo = 0.f, hi = 0.f;
        if (h == 0) {
            for (int j = 0; j < k; ++j) {
                const float cv = sm.cin[j * CS + k];
                lo += fminf(cv, 0.f);
                hi += fmaxf(cv, 0.f);
            }
            sm.lo_i[k] = lo;
            sm.hi_i[k] = hi;
        } else {
            if (c.win)
                for (int j = 0; j < c.nwk; ++j) {
                    const float cv = sm.cwin[j * CS + k];
                    lo += fminf(cv, 0.f);
                    hi += fmaxf(cv, 0.f);
                }
            sm.lo_w[k] = lo;
            sm.hi_w[k] = hi;
            // 3a. the move's own part of step 3, which needs no tile: far-field bound coefficients, the band of
            // the overlap test, and the overlap status from this group's and the window's ions (the deep
            // windows' becomes exact after the tiles)
            unsigned stv = sm.st[k];
            const float4 ak = sm.trial[k], bk = sm.own[k];
            const float dx = ak.x - bk.x, dy = ak.y - bk.y, dz = ak.z - bk.z;
            const float dn = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) * (1.0f + 0x1p-18f);
            float kT = 0.f, kP = 0.f, kO = 0.f;
            const bool bounded = far_coeffs(dn, sp, kT, kP, kO);
            sm.kTs[k] = bounded ? kT : -1.f;
            // P's coefficient also carries the tiles' |t| terms: |t| <= dn rn ro (triangle inequality), with
            // slack for the rounding of the computed rn ro
            sm.kPs[k] = kP + (C_SUM + kT + 0x1p-12f) * dn * (1.0f + 0x1p-16f);
            // the settled ions' squared distances come from pair_far: widen the overlap band to its error
            const float rel = kO * U32;
            sm.lo2ks[k] = fminf(lo2, s2f * (1.0f - rel) * (1.0f - 0x1p-22f));
            sm.hi2ks[k] = fmaxf(hi2, s2f * (1.0f + rel) * (1.0f + 0x1p-22f));
            if (!(stv & (ST_INACTIVE | ST_WALL))) {
                if (!bounded) stv |= ST_OVL_AMBIG;
                unsigned any = 0, both = 0;
#pragma unroll
                for (int w = 0; w < WORDS; ++w) {
                    any |= sm.ovo[k][w] | sm.ovn[k][w] | sm.wovo[k][w] | sm.wovn[k][w];
                    both |= (sm.ovo[k][w] & sm.ovn[k][w]) | (sm.wovo[k][w] & sm.wovn[k][w]);
#pragma unroll
                    for (int d = 0; d < DW; ++d) both |= sm.dovo[d][k][w] & sm.dovn[d][k][w];
                    any |= sm.dovo[0][k][w] | sm.dovn[0][k][w];  // deep window 0 is exact only at step 5
                }
                if (both) stv |= ST_OVL_CERTAIN;
                else if (any) stv |= ST_OVL_POSSIBLE;
                sm.st[k] = (unsigned char)stv;
            }
            sm.bnd[k] = finf();  // moves without pair sums keep it
            sm.run[k] = 0.f;
            sm.wex[k] = 0.f;
        }
    }
    // the deep-window pass's partials join slice 0's accumulators of each slot (its barrier is 2b''s)
    if (c.nd > 0 && r == 0) {
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            if (km[m] < 0) continue;
            const int n = p + 32 * m;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float s2, e;
                two_sum(hA[m], sm.dsh[hh][n], s2, e);
                hA[m] = s2;
                lA[m] = lA[m] + sm.dsl[hh][n] + e;
                AA[m] += sm.dsA[hh][n];
                TA[m] += sm.dsT[hh][n];
                CA[m] += sm.dsC[hh][n];
            }
        }
    }
    }  // !helper
    // 2c. every other group, oldest published version first (Algorithm 2 per guest group):
    // J = g+1 .. B-1 (version s-1), then J = 0 .. g-1 (version s), the window excluded.
    // In pairs mode each CTA of the cluster takes every other group of this order (leader even, helper odd).
    const int tstep = pairs ? 2 : 1, toff = helper ? 1 : 0;
    const int ntl_all = (B - 1) - (c.win ? 1 : 0) - c.nd;  // the windows are the last groups in this order
    const int ntl = ntl_all > toff ? (ntl_all - toff + tstep - 1) / tstep : 0;
    auto tile_J = [&](int i) -> int { return (g + 1 + tstep * i + toff) % B; };
    auto tile_tag = [&](int J) -> unsigned { return J > g ? tag_prev : tag_cur; };
    auto tile_src = [&](int J) -> const float4 * { return (J > g ? c.Pprev : c.Pcur) + (size_t)J * S; };
    auto tile_words = [&](int J) -> int { return (min(S, N - J * S) + 31) / 32; };
    const long long cyc_t0 = clock64();
    // Publication horizon: tiles 0..hz are known to be published and covered by an acquire fence.  Warp 0
    // polls word 0 of the next 32 tiles (one relaxed load per lane); a single fence covers every newly
    // confirmed tile, so old versions cost no per-tile synchronisation.  The horizon lives in two slots:
    // iteration i reads slot i&1 (written before the barrier that ended iteration i-1) and warp 0 writes
    // slot (i+1)&1, so every thread of an iteration sees the same value.
    auto advance_horizon = [&](int from) -> int {  // warp 0, all lanes; returns the new horizon
        const int t = from + 1 + lane;
        bool ready = false;
        if (t < ntl) {
            const int J = tile_J(t);
            ready = (unsigned)(ld_relaxed(&ch.flags[J * WORDS]) >> 32) == tile_tag(J);
        }
        const unsigned bal = __ballot_sync(FULL, ready);
        const int run = __ffs(~bal) - 1;  // consecutive ready tiles after `from` (-1: all 32)
        const int hz = min((run < 0) ? from + 32 : from + run, ntl - 1);
        if (hz > from) fence_acq_rel();
        return hz;
    };
    // Tiles are staged in pairs where both groups lie inside the publication horizon, so most barriers cover
    // 256 ions; otherwise one group.  Buffer b (iteration parity) holds tcnt[b] groups and horizon hzs[b].
    if (ntl > 0 && ns > 0) {
        if (warp == 0) {
            int hz0 = advance_horizon(-1);
            bool ok = true;
            if (hz0 < 0) {  // the oldest tile is not published yet: wait for it
                const int J0 = tile_J(0);
                unsigned bits;
                ok = wait_words(ch, J0, tile_words(J0), tile_tag(J0), tile_tag(J0), ctl, bits, true, false, SHG);
                hz0 = 0;
            }
            if (lane == 0) {
                sm.ok = ok;
                sm.hzs[0] = hz0;
                sm.tcnt[0] = next_groups(0, ntl, hz0);
            }
        }
        bar_main();
        if (!sm.ok) return false;
#pragma unroll
        for (int u = 0; u < TG * S / T; ++u) {
            const int q = u * T + tid;
            if (q < sm.tcnt[0] * S) sm.tile[0][q] = __ldcg(&tile_src(tile_J(q >> 7))[q & (S - 1)]);
        }
        bar_main();
    }
    // the tiles run two moves per packed FP32x2 instruction (slots (0,1) and (2,3)); their |t| sum is bounded
    // by dn P instead of accumulated
    Mv2 mv[MPT / 2];
    f32x2 s2[MPT / 2], P2[MPT / 2];
#pragma unroll
    for (int pp = 0; pp < MPT / 2; ++pp) {
        const int m0 = 2 * pp, m1 = 2 * pp + 1;
        mv[pp] = make_mv2(b3[m0], d3[m0], b3[m1], d3[m1]);
        s2[pp] = pk2(sA[m0], sA[m1]);
        P2[pp] = pk2(PA[m0], PA[m1]);
    }
    // excess mode (65..72 occupied slots, delayed acceptance or the prefilter, no helper warps, no pairs): two layers
    // as usual and the e = ns - 64 excess moves by 8 rows of 32 threads (tile_buffer_x), instead of a third layer of
    // 32 move slots that would cost half as much again as the two
    const int nex = ns - 64;
    const int XS = (DA && !HELP && !pairs && nex > 0 && nex <= 8) ? 32 : 0;
    const int qx = XS ? tid / XS : 0, rx = XS ? tid % XS : 0;
    const bool xact = XS && qx < nex;
    Mv2 mx;
    float sx = 0.f, Px = 0.f, mnx = finf(), hx = 0.f, lx = 0.f;
    {
        const int kx = (int)sm.surv[xact ? 64 + qx : 0];
        const float4 ax = sm.trial[kx], bx = sm.own[kx];
        const float3 bx3 = make_float3(bx.x, bx.y, bx.z), dx3 = make_float3(ax.x - bx.x, ax.y - bx.y, ax.z - bx.z);
        mx = make_mv2(bx3, dx3, bx3, dx3);
    }
    // with helper warps: hand the tile pass over (they wait at barrier 2); they take column slices 8..15
    const bool tiles_run = ntl > 0 && ns > 0;
    if (HELP) {
        if (tid == 0) {
            sm.hcmd[hseq & 1] = tiles_run ? HC_RUN : HC_SKIP;
            sm.hntl[hseq & 1] = ntl;
        }
        ++hseq;
        bar_all();
    }
    auto tile_bar = [&]() {
        if (HELP) bar_all();
        else bar_main();
    };
    int it = 0;
    for (int i = 0; tiles_run && i < ntl; ++it) {
        const int cur = it & 1;
        const int cnt = sm.tcnt[cur];
        const int hz = sm.hzs[cur];
        const int in = i + cnt;  // first group of the next buffer
        const int pn = next_groups(in, ntl, hz);  // groups prefetched
        // the next buffer's groups are copied into the other buffer (16 B per thread and copy, through L2) while
        // this one runs; the copies complete before the barrier that ends the iteration
#pragma unroll
        for (int u = 0; u < TG * S / T; ++u) {
            const int q = u * T + tid;
            if (q < pn * S) cp_async16(&sm.tile[cur ^ 1][q], &tile_src(tile_J(in + (q >> 7)))[q & (S - 1)]);
        }
        // occupied 32-move layers only (all of them for a plain chain)
        if (XS == 32)
            tile_buffer_x<32>(sm.tile[cur], cnt, r, mv[0], s2[0], P2[0], mA[0], mA[1], hA[0], lA[0], hA[1], lA[1], xact,
                              rx, mx, sx, Px, mnx, hx, lx);
        else
            tile_buffer<HELP ? 2 * SL : SL>(sm.tile[cur], cnt, r, nm, mv, s2, P2, mA, hA, lA);
        cp_async_wait_all();
        if (warp == 0) {
            const int nh = (hz < in + 4 * TG && hz < ntl - 1) ? advance_horizon(hz) : hz;
            if (lane == 0) {
                sm.hzs[cur ^ 1] = nh;
                sm.tcnt[cur ^ 1] = pn;
            }
        }
        tile_bar();
        if (in < ntl && pn == 0) {  // the next tile was not published in time: wait for it now (uniform branch)
            const int Jn = tile_J(in);
            if (warp == 0) {
                unsigned bits;
                const bool ok = wait_words(ch, Jn, tile_words(Jn), tile_tag(Jn), tile_tag(Jn), ctl, bits, true, false, SHG);
                if (lane == 0) {
                    sm.ok = ok;
                    sm.hzs[cur ^ 1] = max(sm.hzs[cur ^ 1], in);
                    sm.tcnt[cur ^ 1] = 1;
                }
            }
            tile_bar();
            if (!sm.ok) return false;
            if (trc) gt_tile = globaltimer();
            if (tid < S) sm.tile[cur ^ 1][tid] = __ldcg(&tile_src(Jn)[tid]);
            tile_bar();
        }
        i = in;
    }
    if (HELP && tiles_run) bar_all();  // the helpers' per-move sums are in shared memory
    if (XS) {  // excess moves: combine each row's XS slices (a warp or half a warp) and hand the sums over
        for (int o = 1; o < XS; o <<= 1) {
            const float h2 = __shfl_xor_sync(FULL, hx, o), l2 = __shfl_xor_sync(FULL, lx, o);
            float t2, e;
            two_sum(hx, h2, t2, e);
            hx = t2;
            lx = lx + l2 + e;
            Px += __shfl_xor_sync(FULL, Px, o);
            mnx = fminf(mnx, __shfl_xor_sync(FULL, mnx, o));
        }
        if (xact && rx == 0) {
            const int kx = sm.surv[64 + qx];
            help_h(sm)[kx] = hx;
            help_l(sm)[kx] = lx;
            help_p(sm)[kx] = Px;
            help_m(sm)[kx] = mnx;
        }
        bar_main();
    }
    cyc_tiles = clock64() - cyc_t0;
    if (trc) gt_tiles = globaltimer();
#pragma unroll
    for (int pp = 0; pp < MPT / 2; ++pp) upk2(P2[pp], PA[2 * pp], PA[2 * pp + 1]);
    PairBox *const box = pairs ? &ctl->box[blockIdx.x >> 1] : nullptr;
    if (helper) {
        // combine the slices and hand the per-move tile sums to the leader
#pragma unroll
        for (int o = 1; o < SL; o <<= 1) {
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                const float h2 = __shfl_xor_sync(FULL, hA[m], o), l2 = __shfl_xor_sync(FULL, lA[m], o);
                float s2, e;
                two_sum(hA[m], h2, s2, e);
                hA[m] = s2;
                lA[m] = lA[m] + l2 + e;
                PA[m] += __shfl_xor_sync(FULL, PA[m], o);
                mA[m] = fminf(mA[m], __shfl_xor_sync(FULL, mA[m], o));
            }
        }
        if (r == 0) {
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                const int k = km[m];
                if (k < 0) continue;
                __stcg(&box->h[k], hA[m]);
                __stcg(&box->l[k], lA[m]);
                __stcg(&box->p[k], PA[m]);
                __stcg(&box->m[k], mA[m]);
            }
        }
        cluster_sync_all();  // hand-over to the leader
        return true;
    }
    if (pairs) {
        cluster_sync_all();  // the helper's tile sums are in the box
        if (tid == 0) sm.ok = *(volatile int *)&ctl->abort ? 0 : 1;
        bar_main();
        if (!sm.ok) return false;
    }

    // 2d. combine the 8 column slices (warp-local) into the float-float sum, one bound sum (the bound's linear
    // combination of the magnitude sums, all coefficients positive) and the minimum squared distance, while
    // warp 0 reads the deep windows' outcome words (one contiguous run of groups); then the deep windows' exact
    // correction sums and overlap bits from TMEM.  The bound sums carry FP32 rounding of at most n u relative
    // for n terms per thread: infl covers it.
    const float infl = 1.0f + (float)(N / SL + 64 * DW + 64) * 0x1p-23f;
    bar_main();  // 3a's per-move coefficients (no tile loop may have run since)
    float QA[MPT];
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        const float kT = sm.kTs[km[m] < 0 ? 0 : km[m]], kP = sm.kPs[km[m] < 0 ? 0 : km[m]];
        QA[m] = (kT < 0.f) ? finf()
                           : C_TERM * AA[m] + (C_SUM + kT + 0x1p-12f) * TA[m] + kP * PA[m] + C_CORR * CA[m];
    }
#pragma unroll
    for (int o = 1; o < SL; o <<= 1) {
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const float h2 = __shfl_xor_sync(FULL, hA[m], o), l2 = __shfl_xor_sync(FULL, lA[m], o);
            float s2, e;
            two_sum(hA[m], h2, s2, e);
            hA[m] = s2;
            lA[m] = lA[m] + l2 + e;
            QA[m] += __shfl_xor_sync(FULL, QA[m], o);
            mA[m] = fminf(mA[m], __shfl_xor_sync(FULL, mA[m], o));
        }
    }
    if (r < MPT) {  // lane r of each slice group stores move slot m = r (every lane holds the combined values)
        float hv = hA[0], lv = lA[0], qv = QA[0], mv = mA[0];
        int kv = km[0];
#pragma unroll
        for (int m = 1; m < MPT; ++m)
            if (r == m) {
                hv = hA[m];
                lv = lA[m];
                qv = QA[m];
                mv = mA[m];
                kv = km[m];
            }
        if (kv >= 0) {
            if (pairs) {  // the helper's tiles
                float s2, e;
                two_sum(hv, __ldcg(&box->h[kv]), s2, e);
                hv = s2;
                lv = lv + __ldcg(&box->l[kv]) + e;
                qv += sm.kPs[kv] * __ldcg(&box->p[kv]);
                mv = fminf(mv, __ldcg(&box->m[kv]));
            }
            if ((HELP && tiles_run) || (XS && r == 2)) {  // the helper warps' column slices, or the excess rows
                float s2, e;
                two_sum(hv, help_h(sm)[kv], s2, e);
                hv = s2;
                lv = lv + help_l(sm)[kv] + e;
                qv += sm.kPs[kv] * help_p(sm)[kv];
                mv = fminf(mv, help_m(sm)[kv]);
            }
            sm.bhi[kv] = hv;
            sm.blo[kv] = lv;
            sm.Qs[kv] = qv;
            sm.mind2[kv] = mv;
        }
    }
    if (c.nd > 1) {  // deep windows 1.. (published at least two group-times before the window)
        if (warp == 0) {
            unsigned bits;
            const int nw = (c.nd - 1) * WORDS;
            const bool ok = wait_words(ch, g - 1 - c.nd, nw, tag_cur, tag_cur, ctl, bits, false, true, SHG);
            if (lane < nw) sm.dacc[c.nd - 1 - lane / WORDS][lane % WORDS] = bits;
            if (lane == 0) sm.ok = ok;
        }
        bar_main();
        if (!sm.ok) return false;
        const int q = warp & 3, h = warp >> 2, n = 32 * q + lane;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};  // independent partial sums
        unsigned wo = 0u;
        if (32 * q < ns) {  // warp-uniform
            const int k = sm.surv[n < ns ? n : 0];
            for (int d = 1; d < c.nd; ++d) {
#pragma unroll
                for (int q32 = 0; q32 < HALF / 32; ++q32) {
                    float v[32];
                    __syncwarp();
                    tmem_ld32(tbase + (unsigned)(S * d + h * HALF + 32 * q32), v);
                    const int w = 2 * h + q32;
                    const unsigned wb = sm.dacc[d][w];
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[i & 3] += ((wb >> i) & 1u) ? v[i] : 0.f;
                    wo |= (sm.dovn[d][k][w] & wb) | (sm.dovo[d][k][w] & ~wb);
                }
            }
        }
        sm.dpart[h][n] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        sm.dwo[h][n] = wo;
    }
    bar_main();
    if (trc) gt_ph[0] = globaltimer();

    // 3b + 4. per move: the deep windows' exact sums and overlap, the settled ions' overlap from the minimum
    // squared distance, the static FP32 band; then round 0: moves decided whatever the window and this group's
    // earlier moves do
    if (tid < S) {
        const int k = tid;
        unsigned stv = sm.st[k];
        const int n = sm.slot[k];
        if (n != 255) {
            const float kT = sm.kTs[k];
            if (c.nd > 1) {
                sm.wexd[k] = sm.dpart[0][n] + sm.dpart[1][n];
                if (sm.dwo[0][n] | sm.dwo[1][n]) stv |= ST_OVL_CERTAIN;
            }
            if (!(stv & (ST_INACTIVE | ST_WALL)) && kT >= 0.f) {
                const float m2 = sm.mind2[k];
                if (m2 < sm.lo2ks[k]) stv |= ST_OVL_CERTAIN;
                else if (!(m2 > sm.hi2ks[k])) stv |= ST_OVL_AMBIG;
            }
            sm.st[k] = (unsigned char)stv;
            const float lqa = fabsf(lBf * sm.own[k].w);
            float bnd = (mode == 1 || mode == 3 || kT < 0.f)
                            ? finf()
                            : (mode == 2 ? 0.f : lqa * (U32 * (sm.Qs[k] * infl) + 0x1p-40f * ch.a_max));
            if (DA && ch.da && !ch.pf && mode == 0) bnd += sm.dEtB[k];  // stage 2 compares dE with L(u2) + dEt
            sm.bnd[k] = bnd;
        }
        if (trc) gt_ph[1] = globaltimer();
        int out = -1;
        if (stv & ST_INACTIVE) out = OUT_INACTIVE;
        else if (stv & ST_WALL) out = OUT_WALL;
        else if (stv & ST_DA_DONE) out = sm.outcome[k];
        else if (stv & ST_OVL_CERTAIN) out = OUT_OVERLAP;
        else if (!(stv & (ST_OVL_POSSIBLE | ST_OVL_AMBIG))) {
            if (stv & ST_UZERO) out = OUT_ACCEPT;
            else {
                const float lq = lBf * sm.own[k].w;
                const float base = sm.bhi[k] + sm.blo[k];
                const int n0 = sm.slot[k];
                const float l0 = (c.nd > 0 && n0 != 255) ? sm.dlo[0][n0] + sm.dlo[1][n0] : 0.f;
                const float h0 = (c.nd > 0 && n0 != 255) ? sm.dhi[0][n0] + sm.dhi[1][n0] : 0.f;
                out = decide_interval(sm, k, lq, base + ((sm.lo_w[k] + (sm.wexd[k] + l0)) + sm.lo_i[k]),
                                      base + ((sm.hi_w[k] + (sm.wexd[k] + h0)) + sm.hi_i[k]));
            }
        }
        if (out >= 0 && out <= OUT_DA1) sm.outcome[k] = (signed char)out;
        const unsigned dec = __ballot_sync(FULL, out >= 0);
        const unsigned acc = __ballot_sync(FULL, out == OUT_ACCEPT);
        if (lane == 0) {
            sm.decw[warp] = dec;
            sm.accw[warp] = acc;
        }
    }

    // 5. first in-group partial pass (needs only round 0's decisions), then the window's outcome (the
    // critical wait) and its exact correction sums.
    bar_main();
    if (trc) gt_ph[2] = globaltimer();
    if (tid < WORDS) {
        sm.acc0[tid] = sm.accw[tid];
        sm.dec0[tid] = sm.decw[tid];
    }
    bar_main();
    partial_pass(sm);
    if (trc) gt_ready = globaltimer();
    const long long cyc_w0 = clock64();
    if (c.nd > 0) {
        // deep window 0 (the group before the window, published a group-time before it): its exact correction
        // sums from TMEM and its exact overlap
        if (warp == 0) {
            unsigned bits;
            const bool ok = wait_words(ch, g - 2, WORDS, tag_cur, tag_cur, ctl, bits, false, true, SHG);
            if (lane < WORDS) sm.dacc[0][lane] = bits;
            if (lane == 0) sm.ok = ok;
        }
        bar_main();
        if (!sm.ok) return false;
        if (trc) gt_w2 = globaltimer();
        {
            const int q = warp & 3, h = warp >> 2, n = 32 * q + lane;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            unsigned wo = 0u;
            if (32 * q < ns) {  // warp-uniform
                const int k = sm.surv[n < ns ? n : 0];
#pragma unroll
                for (int q32 = 0; q32 < HALF / 32; ++q32) {
                    float v[32];
                    __syncwarp();
                    tmem_ld32(tbase + (unsigned)(h * HALF + 32 * q32), v);
                    const int w = 2 * h + q32;
                    const unsigned wb = sm.dacc[0][w];
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[i & 3] += ((wb >> i) & 1u) ? v[i] : 0.f;
                    wo |= (sm.dovn[0][k][w] & wb) | (sm.dovo[0][k][w] & ~wb);
                }
            }
            sm.dpart[h][n] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            sm.dwo[h][n] = wo;
        }
        bar_main();
        if (tid < ns) {
            const int n = tid, k = sm.surv[n];
            sm.wexd[k] += sm.dpart[0][n] + sm.dpart[1][n];
            if (sm.dwo[0][n] | sm.dwo[1][n]) sm.st[k] = (unsigned char)(sm.st[k] | ST_OVL_CERTAIN);
        }
    }
    if (c.win) {
        if (warp == 0) {
            unsigned bits;
            const int nw = (c.nwk + 31) / 32;
            const bool ok = wait_words(ch, c.Jw, nw, (unsigned)(sw + 1), (unsigned)(sw + 1), ctl, bits, false, true, SHG);
            if (lane < WORDS) sm.winacc[lane] = (lane < nw) ? bits : 0u;
            if (lane == 0) sm.ok = ok;
        }
        bar_main();
        if (!sm.ok) return false;
        cyc_win = clock64() - cyc_w0;
        if (trc) gt_window = globaltimer();
        cw0 = clock64();
        {
            const int k = tid & (S - 1), h = tid >> 7;
            float sx = 0.f;
            const unsigned wa0 = sm.winacc[2 * h], wa1 = sm.winacc[2 * h + 1];
            const float *col = &sm.cwin[(h * HALF) * CS + k];
            // four independent partial sums over batches of 16 loads issued together
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int jb = 0; jb < HALF; jb += 16) {
                const unsigned wb = (jb < 32 ? wa0 : wa1) >> (jb & 31);
                float cv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) cv[u] = col[(jb + u) * CS];
#pragma unroll
                for (int u = 0; u < 16; ++u) acc[u & 3] += ((wb >> u) & 1u) ? cv[u] : 0.f;
            }
            sx = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            sm.wpart[h][k] = sx;
        }
        bar_main();
        cres[0] = (unsigned)(clock64() - cw0);
        if (tid < S) {
            const int k = tid;
            sm.wex[k] = (sm.wpart[0][k] + sm.wpart[1][k]) + sm.wexd[k];
            unsigned wo = 0;  // the window's overlap is now exact
#pragma unroll
            for (int w = 0; w < WORDS; ++w) wo |= (sm.wovn[k][w] & sm.winacc[w]) | (sm.wovo[k][w] & ~sm.winacc[w]);
            if (wo) sm.st[k] = (unsigned char)(sm.st[k] | ST_OVL_CERTAIN);
        }
    }
    bar_main();
    cres[1] = (unsigned)(clock64() - cw0);

    // 6. rounds over this group's earlier moves: exact sums over decided ones,
    // intervals over undecided ones.  The first undecided move has only decided
    // predecessors after at most one more round; if it is still inside its band
    // it goes to the guard tiers.
    cyc_res0 = clock64();
    for (;;) {
        ++n_rounds;
        if (tid < S) {
            const int k = tid;
            int out = -1;
            if (!bit(sm.dec0, k)) {
                const float run = sm.run[k] + (sm.part[0][k] + sm.part[1][k]);
                sm.run[k] = run;
                const float lo = sm.plo[0][k] + sm.plo[1][k], hi = sm.phi[0][k] + sm.phi[1][k];
                const unsigned stv = sm.st[k];
                bool ov_c, ov_p;
                ingroup_overlap(sm, k, sm.dec0, sm.acc0, ov_c, ov_p);
                bool unknown = false;
#pragma unroll
                for (int w = 0; w < WORDS; ++w) unknown |= (~sm.dec0[w] & below(k, w)) != 0u;
                if ((stv & ST_OVL_CERTAIN) || ov_c) out = OUT_OVERLAP;
                else if (!ov_p && !(stv & ST_OVL_AMBIG)) {
                    if (stv & ST_UZERO) out = OUT_ACCEPT;
                    else {
                        const float lq = lBf * sm.own[k].w;
                        const float base = sm.bhi[k] + (sm.blo[k] + (sm.wex[k] + run));
                        out = decide_interval(sm, k, lq, base + lo, base + hi);
                    }
                }
                if (out >= 0) {
                    sm.outcome[k] = (signed char)out;
                    sm.tier[k] = unknown ? 0 : 1;
                }
            }
            const unsigned dec = __ballot_sync(FULL, out >= 0);
            const unsigned acc = __ballot_sync(FULL, out == OUT_ACCEPT);
            if (lane == 0) {
                sm.seen[warp] = sm.acc0[warp];
                sm.decw[warp] |= dec;
                sm.accw[warp] |= acc;
            }
        }
        bar_main();
        if (n_rounds == 1) cres[2] = (unsigned)(clock64() - cw0);
        cres[3] = (unsigned)(clock64() - cw0);
        int first = -1;
#pragma unroll
        for (int w = 0; w < WORDS; ++w) {
            const unsigned und = ~sm.decw[w];
            if (first < 0 && und) first = w * 32 + __ffs(und) - 1;
        }
        if (first < 0 || first >= nk) break;
        bool exact = true;  // were all predecessors of `first` decided when this round started?
#pragma unroll
        for (int w = 0; w < WORDS; ++w) exact &= (~sm.dec0[w] & below(first, w)) == 0u;
        if (exact) {
            // guard tiers on move k = first: exact FP32 value was inside its band (or overlap was ambiguous)
            const long long cyc_g0 = clock64();
            const int k = first;
            const unsigned stv = sm.st[k];
            // the acceptance draw of this decision: purpose 0, or purpose 1 for delayed acceptance's stage 2
            const bool isda = DA && ch.da != nullptr && !ch.pf;
            const unsigned ua =
                move_draws(ch, s * (unsigned long long)N + (unsigned long long)(k0 + k), isda ? 1u : 0u).w >> 8;
            const double L64 = (ua == 0u) ? 0.0 : -series_log((double)ua * 0x1p-24);
            if ((stv & ST_OVL_AMBIG) && mode != 1) {
                // settle the overlap question first; without an overlap the move is decided by the next round
                const long long q0 = clock64();
                const bool ov = overlap_exact(sm, c, k);
                cyc_ovl += clock64() - q0;
                ++n_scan;
                if (tid == 0) {
                    if (ov) {
                        sm.outcome[k] = (signed char)OUT_OVERLAP;
                        sm.tier[k] = 5;
                        sm.decw[k >> 5] |= 1u << (k & 31);
                    } else {
                        sm.st[k] = (unsigned char)(stv & ~ST_OVL_AMBIG);
                    }
                }
            } else {
                double dE = 0.0;
                int res = -1, tier = 2;
                // delayed acceptance compares fl(dE - dEt) with L(u2): the reference dEt, and the threshold for dE
                double dEt64 = 0.0, thr = L64, xs = 0.0;
                if (isda) {
                    if (!bit(sm.d64w, k)) {
                        const double v = da_dEt64(sm, c, k);
                        ++n_dfp64;
                        if (tid == 0) {
                            sm.dEt64[k] = v;
                            sm.d64w[k >> 5] |= 1u << (k & 31);
                        }
                        bar_main();
                    }
                    dEt64 = sm.dEt64[k];
                    thr = __dadd_rn(L64, dEt64);
                    xs = 0x1p-50 * (fabs(L64) + fabs(dEt64));
                }
                if (!(stv & ST_OVL_AMBIG) && mode != 1) {
                    long long q0 = clock64();
                    res = SHG ? gb_tier(sm, c, ctl, k, 2, thr, xs, dE) : -2;
                    if (res == -2) res = tier2(sm, c, k, thr, xs, dE);
                    cyc_t[0] += clock64() - q0;
                    if (res < 0) {
                        tier = 3;
                        q0 = clock64();
                        res = SHG ? gb_tier(sm, c, ctl, k, 3, thr, xs, dE) : -2;
                        if (res == -2) res = tier3(sm, c, k, thr, xs, dE);
                        cyc_t[1] += clock64() - q0;
                    }
                }
                if (res < 0) {
                    bool ovl = false;
                    tier = 4;
                    const long long q0 = clock64();
                    tier4(sm, c, k, dE, ovl);
                    cyc_t[2] += clock64() - q0;
                    if (ovl) res = 2;
                    else if (ua == 0u) res = 0;
                    else res = ((isda ? __dsub_rn(dE, dEt64) : dE) < L64) ? 0 : 1;
                }
                if (tid == 0) {
                    const int out = res == 0 ? OUT_ACCEPT : (res == 1 ? OUT_METROPOLIS : OUT_OVERLAP);
                    sm.outcome[k] = (signed char)out;
                    sm.tier[k] = (unsigned char)tier;
                    sm.dEv[k] = dE;
                    sm.decw[k >> 5] |= 1u << (k & 31);
                    if (out == OUT_ACCEPT) sm.accw[k >> 5] |= 1u << (k & 31);
                }
            }
            bar_main();
            cyc_guard += clock64() - cyc_g0;
        } else {
            // every thread must have read dec0 for `exact` before it is overwritten below: a warp that read the
            // new value would find `first` ready, take the guard tiers' barriers alone and fall out of step
            bar_main();
        }
        if (tid < WORDS) {
            sm.acc0[tid] = sm.accw[tid];
            sm.dec0[tid] = sm.decw[tid];
        }
        bar_main();
        partial_pass(sm);
    }
    const long long cyc_resolve = clock64() - cyc_res0 - cyc_guard;
    if (trc) gt_resolved = globaltimer();
    cres[4] = (unsigned)(clock64() - cw0);
    cres[7] = (unsigned)n_rounds;

    // 7. publish: the outcome words first (the next group holds both candidate positions and needs only
    // these bits), then the final positions (version s) and their release-stored words.
    const bool publish = (long long)ticket != ctl->skip_ticket;
    if (warp == 0 && publish && lane < (nk + 31) / 32)
        st_relaxed(&ch.bits[g * WORDS + lane], ((unsigned long long)tag_cur << 32) | sm.accw[lane]);
    if (trc) gt_pub = globaltimer();
    cres[5] = (unsigned)(clock64() - cw0);
    if (tid < nk) {
        const bool acc = bit(sm.accw, tid);
        __stcg(&ch.pos[(s + 1) & 1][k0 + tid], acc ? sm.trial[tid] : sm.own[tid]);
        if (DA && ch.da && acc && publish) {
            // delayed acceptance and the prefilter: the near-field cell list holds current positions (an ion
            // left out of a full prefilter cell has no slot)
            const DADev &dd = *ch.da;
            const int sl = __ldg(&dd.slot_of[k0 + tid]);
            const float4 tv = sm.trial[tid];
            if (sl >= 0) __stcg(&dd.cell_pos[sl], ch.pf ? make_float4(tv.x, tv.y, tv.z, __int_as_float(k0 + tid)) : tv);
        }
    }
    bar_main();
    if (warp == 0 && publish && lane < (nk + 31) / 32)  // release after the barrier: orders every thread's stores
        st_release(&ch.flags[g * WORDS + lane], ((unsigned long long)tag_cur << 32) | sm.accw[lane]);
    const unsigned long long gt_posp = trc ? globaltimer() : 0ull;
    cres[6] = (unsigned)(clock64() - cw0);
    if (tid == 0 && ch.trace) {
        const unsigned long long item = s * (unsigned long long)B + (unsigned long long)g;
        const unsigned long long idx = item - ch.rec_sweep0 * (unsigned long long)B;
        if (item >= ch.rec_sweep0 * (unsigned long long)B && idx < (unsigned long long)ch.trace_cap) {
            TraceRec tr;
            tr.item = item;
            tr.t_start = gt_start;
            tr.t_ready = gt_ready;
            tr.t_window = gt_window;
            tr.t_resolved = gt_resolved;
            tr.t_published = gt_pub;
            tr.n_guard = (unsigned long long)(cyc_guard > 0);
            tr.t_positions = gt_posp;
            tr.t_tile = gt_tile;
            tr.t_tiles = gt_tiles;
            tr.t_w2 = gt_w2;
#pragma unroll
            for (int q = 0; q < 4; ++q) tr.t_ph[q] = gt_ph[q];
#pragma unroll
            for (int q = 0; q < 8; ++q) tr.c_res[q] = cres[q];
            ch.trace[idx] = tr;
        }
    }

    // 8. off the critical path: FP32 dE of every evaluated move, ledger, counters, records
    {
        const int k = tid & (S - 1), h = tid >> 7;
        float sx = 0.f;
        const int j0 = h * HALF, j1 = min(k, j0 + HALF);
        for (int j = j0; j < j1; ++j)
            if (bit(sm.accw, j)) sx += sm.cin[j * CS + k];
        sm.part[h][k] = sx;
    }
    bar_main();
    double mydE = 0.0;
    if (tid < S) {
        const int k = tid;
        const int out = sm.outcome[k];
        float d32 = __int_as_float(0x7fc00000);
        if (k < nk && (out == OUT_ACCEPT || out == OUT_METROPOLIS)) {
            const float lq = lBf * sm.own[k].w;
            d32 = lq * (sm.bhi[k] + (sm.blo[k] + (sm.wex[k] + (sm.part[0][k] + sm.part[1][k]))));
            if (sm.tier[k] <= 1) sm.dEv[k] = (double)d32;
        }
        sm.dE32[k] = d32;
        if (k < nk && out == OUT_ACCEPT) mydE = sm.dEv[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mydE += __shfl_xor_sync(FULL, mydE, o);
    if (lane == 0) sm.redd[warp] = mydE;
    bar_main();
    if (tid == 0 && publish) {
        double gsum = 0.0;
        for (int w = 0; w < T / 32; ++w) gsum += sm.redd[w];
        const unsigned long long me = s * (unsigned long long)B + (unsigned long long)g;
        unsigned long long t0 = 0;  // started at the first check
        unsigned spins = 0;
        bool ok = true;
        while (ld_acquire(ch.ledger_seq) != me) {
            if (*(volatile int *)&ctl->abort) {
                ok = false;
                break;
            }
            if (++spins > 16) __nanosleep(32);
            if ((spins & 63) == 0) {
                const unsigned long long now = globaltimer();
                if (t0 == 0) t0 = now;
                else if ((long long)(now - t0) > ctl->timeout_ns) {
                    atomicCAS(&ctl->err, 0, KERR_TIMEOUT);
                    atomicExch(&ctl->abort, 1);
                    ok = false;
                    break;
                }
            }
        }
        if (ok) {
            volatile double *L = ch.ledger;
            const double e = *L + gsum;
            *L = e;
            // the last group of sweep s folded: e is the total energy after that sweep (Sec. 5.2's E_k)
            if (g == B - 1 && ch.eser && s >= ch.eser_sweep0 && s - ch.eser_sweep0 < (unsigned long long)ch.eser_cap)
                ch.eser[s - ch.eser_sweep0] = e;
            st_release(ch.ledger_seq, me + 1);
        }
        sm.ok = ok ? 1 : 0;
    }
    if (warp == 0) {
        unsigned cnt[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = lane; k < nk; k += 32) {
            const int out = sm.outcome[k], tr = sm.tier[k];
            if (out >= 0 && out <= 3) cnt[out]++;
            if (tr >= 2 && tr <= 5) cnt[4]++;
            if (tr == 0 && (out == OUT_ACCEPT || out == OUT_METROPOLIS)) cnt[5]++;
            if (tr >= 2 && tr <= 4) cnt[4 + tr]++;
            if (out == OUT_DA1) cnt[9]++;
            if (out == OUT_OVERLAP && tr >= 6) cnt[10]++;
        }
#pragma unroll
        for (int q = 0; q < 11; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt[q] += __shfl_xor_sync(FULL, cnt[q], o);
        }
        if (lane == 0) {
            atomicAdd(&ch.stats[CNT_ACCEPT], (unsigned long long)cnt[OUT_ACCEPT]);
            atomicAdd(&ch.stats[CNT_METRO], (unsigned long long)cnt[OUT_METROPOLIS]);
            atomicAdd(&ch.stats[CNT_OVERLAP], (unsigned long long)cnt[OUT_OVERLAP]);
            atomicAdd(&ch.stats[CNT_WALL], (unsigned long long)cnt[OUT_WALL]);
            atomicAdd(&ch.stats[CNT_FP64], (unsigned long long)cnt[4]);
            atomicAdd(&ch.stats[CNT_INTERVAL], (unsigned long long)cnt[5]);
            atomicAdd(&ch.stats[CNT_T2], (unsigned long long)cnt[6]);
            atomicAdd(&ch.stats[CNT_T3], (unsigned long long)cnt[7]);
            atomicAdd(&ch.stats[CNT_T4], (unsigned long long)cnt[8]);
            atomicAdd(&ch.stats[CNT_ROUNDS], (unsigned long long)n_rounds);
            atomicAdd(&ch.stats[CNT_CYC_WIN], (unsigned long long)cyc_win);
            atomicAdd(&ch.stats[CNT_CYC_TILES], (unsigned long long)cyc_tiles);
            atomicAdd(&ch.stats[CNT_CYC_RESOLVE], (unsigned long long)cyc_resolve);
            atomicAdd(&ch.stats[CNT_CYC_GUARD], (unsigned long long)cyc_guard);
            atomicAdd(&ch.stats[CNT_CYC_TOTAL], (unsigned long long)(clock64() - cyc_start));
            atomicAdd(&ch.stats[CNT_CYC_T2], (unsigned long long)cyc_t[0]);
            atomicAdd(&ch.stats[CNT_CYC_T3], (unsigned long long)cyc_t[1]);
            atomicAdd(&ch.stats[CNT_CYC_T4], (unsigned long long)cyc_t[2]);
            if (n_scan) {
                atomicAdd(&ch.stats[CNT_OVL_SCAN], (unsigned long long)n_scan);
                atomicAdd(&ch.stats[CNT_CYC_OVL], (unsigned long long)cyc_ovl);
            }
            if (DA && ch.da) {
                atomicAdd(&ch.stats[CNT_DA_REJ1], (unsigned long long)cnt[9]);
                atomicAdd(&ch.stats[CNT_DA_OVL1], (unsigned long long)cnt[10]);
                atomicAdd(&ch.stats[CNT_DA_FP64], (unsigned long long)n_dfp64);
                atomicAdd(&ch.stats[CNT_CYC_DA1], (unsigned long long)cyc_da);
                for (int q = 0; q < 4; ++q) atomicAdd(&ch.stats[CNT_CYC_DA_PART + q], (unsigned long long)da_part[q]);
            }
        }
    }
    if (ch.rec && s >= ch.rec_sweep0 && tid < nk) {
        const int k = tid;
        const unsigned long long idx = (s - ch.rec_sweep0) * (unsigned long long)N + (unsigned long long)(k0 + k);
        if (idx < (unsigned long long)ch.rec_cap) {
            MoveRec rc;
            rc.m = s * (unsigned long long)N + (unsigned long long)(k0 + k);
            rc.i = k0 + k;
            rc.outcome = sm.outcome[k];
            rc.tier = sm.tier[k];
            rc.pad = 0;
            rc.bound = (double)sm.bnd[k];
            rc.dEt = !(DA && ch.da) ? __longlong_as_double(0x7ff8000000000000ll)
                            : (bit(sm.d64w, k) ? sm.dEt64[k] : (double)sm.dEt32[k]);
            const int out = sm.outcome[k];
            const bool ev = out == OUT_ACCEPT || out == OUT_METROPOLIS;
            rc.dE = ev ? sm.dEv[k] : __longlong_as_double(0x7ff8000000000000ll);
            rc.dE32 = ev ? (double)sm.dE32[k] : __longlong_as_double(0x7ff8000000000000ll);
            ch.rec[idx] = rc;
        }
    }
    bar_main();
    return sm.ok != 0;
}

// The persistent loop of one CTA (T threads); DA: the chains may carry a cell list (delayed acceptance, the
// prefilter).  Plain launches use the instance without it, so its code and registers are the plain path's alone.
template <bool DA>
__device__ __forceinline__ void sweep_body(const ChainDev *__restrict__ chains, const Ticket *__restrict__ sched,
                                           int n_tickets, Ctl *ctl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const bool pairs = ctl->pairs != 0;
    const int role = pairs ? (int)cluster_rank() : 0;
    PairBox *const box = pairs ? &ctl->box[blockIdx.x >> 1] : nullptr;
    for (;;) {
        if (threadIdx.x == 0 && role == 0) {
            const unsigned t = atomicAdd(&ctl->ticket, 1u);
            const int ab = *(volatile int *)&ctl->abort;
            sm.ticket = (ab || t >= (unsigned)n_tickets) ? -1 : (int)t;
            if (pairs) __stcg(&box->ticket, sm.ticket);
        }
        if (pairs) {
            cluster_sync_all();  // the leader's ticket is in the box
            // the helper takes the leader's ticket; after an abort (the leader may have left) it leaves too
            if (threadIdx.x == 0 && role == 1)
                sm.ticket = *(volatile int *)&ctl->abort ? -1 : __ldcg(&box->ticket);
        }
        bar_main();
        const int t = sm.ticket;
        bar_main();
        if (t < 0) break;
        int hseq = 0;
        // uniform: every failure exit follows a barrier
        if (!process_group<false, DA>(sm, chains, sched[t], t, ctl, role, hseq)) break;
    }
    // every exit path releases the TMEM columns before the CTA ends
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(sm.tmem);
}

__global__ void __launch_bounds__(T, 1)
sweep_kernel(const ChainDev *__restrict__ chains, const Ticket *__restrict__ sched, int n_tickets, Ctl *ctl)
{
    sweep_body<false>(chains, sched, n_tickets, ctl);
}

__global__ void __launch_bounds__(T, 1)
sweep_kernel_da(const ChainDev *__restrict__ chains, const Ticket *__restrict__ sched, int n_tickets, Ctl *ctl)
{
    sweep_body<true>(chains, sched, n_tickets, ctl);
}

// The same persistent loop with helper warps: 2T threads, one CTA per SM.  Warpgroups 0-1 (threads < T) run the
// work items exactly as sweep_kernel does, with a larger register budget; warpgroups 2-3 give registers up and only
// take column slices 8..15 of each tile pass (helper_loop), doubling the warps that hide the pair terms' latency.
// Register split (setmaxnreg, per warpgroup): 2 x 128 x HELP_REGS_MAIN + 2 x 128 x HELP_REGS_TILE = 2T x 128, the
// launch's own total, so the increase never waits.  Never used with pairs mode.
constexpr int HELP_REGS_MAIN = 168, HELP_REGS_TILE = 88;
static_assert(HELP_REGS_MAIN + HELP_REGS_TILE == 256 && HELP_REGS_MAIN % 8 == 0 && HELP_REGS_TILE % 8 == 0,
              "register split within the launch's 128 per thread");

__global__ void __launch_bounds__(2 * T, 1)
sweep_kernel_h(const ChainDev *__restrict__ chains, const Ticket *__restrict__ sched, int n_tickets, Ctl *ctl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x >= T) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(HELP_REGS_TILE));
        helper_loop(sm);
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(HELP_REGS_MAIN));
        int hseq = 0;
        for (;;) {
            if (threadIdx.x == 0) {
                const unsigned t = atomicAdd(&ctl->ticket, 1u);
                const int ab = *(volatile int *)&ctl->abort;
                sm.ticket = (ab || t >= (unsigned)n_tickets) ? -1 : (int)t;
            }
            bar_main();
            const int t = sm.ticket;
            bar_main();
            if (t < 0) break;
            if (!process_group<true, true>(sm, chains, sched[t], t, ctl, 0, hseq)) break;
        }
        // release the helper warps (they wait at the next hand-over)
        if (threadIdx.x == 0) sm.hcmd[hseq & 1] = HC_EXIT;
        bar_all();
    }
    // every exit path releases the TMEM columns before the CTA ends
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(sm.tmem);
}

// After a launch of n sweeps: advance every chain's sweep counter.
__global__ void advance_sweeps(const ChainDev *__restrict__ chains, int n_chains, long long n, const Ctl *ctl)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_chains && ctl->err == 0) *chains[c].sweep += (unsigned long long)n;
}

}  // namespace mcg

// Host-side launch wrappers (called from mc_api.cu).
namespace mcg_host {

size_t sweep_smem_bytes()
{
    return sizeof(mcg::Smem);
}

cudaError_t sweep_configure()
{
    cudaError_t e = cudaFuncSetAttribute(mcg::sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(mcg::Smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mcg::sweep_kernel_da, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(mcg::Smem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(mcg::sweep_kernel_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(mcg::Smem));
}

// Resident CTAs of the helper-warp kernel per SM (0 if it cannot run).
cudaError_t sweep_occupancy_h(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcg::sweep_kernel_h, 2 * mcg::T,
                                                         sizeof(mcg::Smem));
}

cudaError_t sweep_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcg::sweep_kernel, mcg::T, sizeof(mcg::Smem));
}

// Clusters of two CTAs that can be resident at once (pairs mode); 0 if the device cannot run them.
cudaError_t sweep_max_clusters(int *n)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(mcg::T);
    cfg.dynamicSmemBytes = sizeof(mcg::Smem);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n, mcg::sweep_kernel, &cfg);
}

cudaError_t sweep_launch(int grid, const mcg::ChainDev *chains, const mcg::Ticket *sched, int n_tickets, mcg::Ctl *ctl,
                         int n_chains, long long n_sweeps, cudaStream_t st, bool pairs, bool help, bool da)
{
    if (help && !pairs) {
        mcg::sweep_kernel_h<<<grid, 2 * mcg::T, sizeof(mcg::Smem), st>>>(chains, sched, n_tickets, ctl);
    } else if (pairs) {  // clusters of two CTAs; grid even
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(mcg::T);
        cfg.dynamicSmemBytes = sizeof(mcg::Smem);
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, mcg::sweep_kernel, chains, sched, n_tickets, ctl);
        if (e != cudaSuccess) return e;
    } else if (da) {
        mcg::sweep_kernel_da<<<grid, mcg::T, sizeof(mcg::Smem), st>>>(chains, sched, n_tickets, ctl);
    } else {
        mcg::sweep_kernel<<<grid, mcg::T, sizeof(mcg::Smem), st>>>(chains, sched, n_tickets, ctl);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mcg::advance_sweeps<<<(n_chains + 127) / 128, 128, 0, st>>>(chains, n_chains, n_sweeps, ctl);
    return cudaGetLastError();
}

}  // namespace mcg_host
