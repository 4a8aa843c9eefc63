// mc_sweep.cu -- the persistent sweep kernel (sm_103a).
//
// What it computes is the sequential-updating Metropolis chain of Sec. 2:
// every sweep tries ions 0..N-1 in order; move i's energy change uses the
// current positions of all other ions (Eq. of the Delta E_ij table: ions
// j < i already at their outcome of this sweep, ions j > i at their position
// from the previous sweep).  How it computes it is GB300-specific:
//
//  * Work items are (chain, group of S = 128 consecutive ions, sweep),
//    handed out in stream order by an atomic ticket, so a CTA only ever waits
//    on work already claimed by a running CTA (no dependence on block
//    dispatch order, which the paper's deadlock argument of Sec. 3.5
//    implicitly assumes).
//  * A CTA computes, for its S moves, the pair sums against every other
//    group's latest published positions, tile by tile (the brush of Sec. 3.4,
//    Algorithm 2), oldest version first; groups publish per-32-ion words
//    ((sweep+1) << 32 | accept bits) with release stores and are read with
//    acquire loads -- a sweep-tagged flag needs no reset (the paper's
//    BlockState array of Algorithm 5 must be cleared by the last block).
//  * Inside the group (Algorithms 3 and 4) the lower-triangle terms are
//    computed for both possible positions of each earlier ion j (old and
//    trial); the correction c_kj = term(trial_j) - term(old_j) is kept in
//    shared memory.  Decisions are then resolved mostly in parallel: a move
//    whose outcome is the same for every combination of the unknown earlier
//    outcomes is decided at once; the rest are decided in order by one warp
//    with exact sums.
//  * Pair terms are FP32 (rsqrt.approx), promoted to FP64 per tile.  A move
//    is decided in FP32 only when |dE + ln u| exceeds a proven bound on the
//    FP32 error; otherwise the whole CTA recomputes dE in the oracle's FP64
//    arithmetic and summation order (the paper computes every energy term in
//    FP64, Sec. 3.3; GB300's FP64 rate makes that the exception here).
//  * Every wait is bounded by %globaltimer; on expiry the kernel records the
//    error, raises an abort flag and all CTAs return.
#include "mc_device.cuh"

namespace mcg {

struct __align__(16) Smem {
    float4 own[S];    // old positions x_k (w = valence)
    float4 trial[S];  // trial positions x'_k (w = valence)
    float4 tile[S];   // one column group
    double Lneg[S];   // -L(u_acc) (+inf when u_acc == 0)
    double base[S];   // FP64 sum of all terms with known positions (+ in-group lower with old positions)
    double dE[S];     // dE of each decided, evaluated move
    float Ab[S];      // sum |q_j| (1/r' + 1/r)  (both versions for in-group lower j)
    float Tb[S];      // sum |t_j| of the terms in base
    float TCb[S];     // sum |c_kj|
    float mind2[S];   // min FP32 |x'_k - x_j|^2 over positions known to be final
    unsigned ovo[S][WORDS];  // bit j: x'_k overlaps old x_j (in-group, j < k)
    unsigned ovn[S][WORDS];  // bit j: x'_k overlaps trial x'_j
    unsigned accw[WORDS];
    unsigned decw[WORDS];
    unsigned char st[S];     // status bits
    signed char outcome[S];
    unsigned char tier[S];
    unsigned char pad0[S];
    float cmat[S * CS];      // c[j][k] at j*CS + k
    double chunk[CHUNK];
    double red[T / 32];
    int ticket;
    int ok;
    int guard_k;
    int ovl_flag;
};

constexpr unsigned ST_WALL = 1u, ST_UZERO = 2u, ST_INACTIVE = 4u, ST_OVL_CERTAIN = 8u, ST_OVL_AMBIG = 16u;
constexpr unsigned FULL = 0xffffffffu;

// Bound constants (units of u = 2^-24); see the error analysis in the design doc.
constexpr double U32 = 0x1p-24;
constexpr double C_TERM = 10.0;   // per-term error of q_j (1/r' - 1/r) relative to |q_j| (1/r' + 1/r)
constexpr double C_SUM = 40.0;    // FP32 partial sums of <= 32 terms before FP64 promotion
constexpr double C_CORR = S + 8;  // FP32 sums of <= S corrections in the resolver

__device__ __forceinline__ bool wait_group(const ChainDev &ch, int J, unsigned need, Ctl *ctl)
{
    const int nw = min(WORDS, (ch.N - J * S + 31) / 32);
    const unsigned long long t0 = globaltimer();
    for (int w = 0; w < nw; ++w) {
        unsigned spins = 0;
        for (;;) {
            const unsigned long long v = ld_acquire(&ch.flags[J * WORDS + w]);
            const unsigned tag = (unsigned)(v >> 32);
            if (tag == need) break;
            if ((int)(tag - need) > 0) {  // a newer version than any reader can need
                atomicCAS(&ctl->err, 0, KERR_PROTOCOL);
                atomicExch(&ctl->abort, 1);
                return false;
            }
            if (*(volatile int *)&ctl->abort) return false;
            if (++spins > 32) __nanosleep(40);
            if ((spins & 63) == 0 && (long long)(globaltimer() - t0) > ctl->timeout_ns) {
                if (atomicCAS(&ctl->err, 0, KERR_TIMEOUT) == 0)
                    ctl->err_info = ((unsigned long long)J << 32) | need;
                atomicExch(&ctl->abort, 1);
                return false;
            }
        }
    }
    return true;
}

// FP32 pair term of move (a = trial, b = old) against y:
// t = q_y (1/|a-y| - 1/|b-y|) accumulated into s; |q|(1/r'+1/r) into A;
// |t| into Tt; |a-y|^2 into the running minimum mn.
__device__ __forceinline__ void pair_acc(const float4 a, const float4 b, const float4 y, float &s, float &A,
                                         float &Tt, float &mn)
{
    const float dxn = a.x - y.x, dyn = a.y - y.y, dzn = a.z - y.z;
    const float d2n = fmaf(dzn, dzn, fmaf(dyn, dyn, dxn * dxn));
    const float dxo = b.x - y.x, dyo = b.y - y.y, dzo = b.z - y.z;
    const float d2o = fmaf(dzo, dzo, fmaf(dyo, dyo, dxo * dxo));
    const float rn = rsqrt_approx(d2n), ro = rsqrt_approx(d2o);
    const float diff = rn - ro;
    s = fmaf(y.w, diff, s);
    A = fmaf(fabsf(y.w), rn + ro, A);
    Tt = fmaf(fabsf(y.w), fabsf(diff), Tt);
    mn = fminf(mn, d2n);
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

// Exact overlap test |a - y|^2 < sigma^2 from the FP32 squared distance, with
// the FP64 squared distance of the FP32 points deciding inside the band.
__device__ __forceinline__ bool overlaps(float d2f, const float4 a, const float4 y, float lo, float hi, double sig2)
{
    if (d2f < lo) return true;
    if (d2f > hi) return false;
    return d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < sig2;
}

// In-group pair (ion j of this group against move k of this group).
__device__ __forceinline__ void ingroup_pair(Smem &sm, int k, int j, const float4 a, const float4 b, const float4 yo,
                                             const float4 yn, float &s, float &A, float &Tt, float &TC, float &mn,
                                             float lo, float hi, double sig2)
{
    if (j > k) {  // ion j moves after k: its old position is final for move k (upper triangle, Algorithm 3)
        pair_acc(a, b, yo, s, A, Tt, mn);
    } else if (j < k) {  // ion j moves before k: position depends on its outcome (Algorithm 4's lower triangle)
        float Ao, An, d2o_n, d2n_n;
        const float to = pair_term(a, b, yo, Ao, d2o_n);
        const float tn = pair_term(a, b, yn, An, d2n_n);
        s += to;
        Tt += fabsf(to);
        A += Ao + An;
        const float c = tn - to;
        sm.cmat[j * CS + k] = c;
        TC += fabsf(c);
        if (overlaps(d2o_n, a, yo, lo, hi, sig2)) atomicOr(&sm.ovo[k][j >> 5], 1u << (j & 31));
        if (overlaps(d2n_n, a, yn, lo, hi, sig2)) atomicOr(&sm.ovn[k][j >> 5], 1u << (j & 31));
    }
}

__device__ __forceinline__ bool bit(const unsigned *w, int j)
{
    return (w[j >> 5] >> (j & 31)) & 1u;
}

// Error bound of the FP32-derived dE of move k ("FP32 error bound").
__device__ __forceinline__ double band(const Smem &sm, int k, double lBabs, int mode)
{
    if (mode == 1) return __longlong_as_double(0x7ff0000000000000ll);  // +inf: always FP64
    if (mode == 2) return 0.0;
    const double A = sm.Ab[k], Tt = sm.Tb[k], TC = sm.TCb[k];
    return lBabs * (U32 * (C_TERM * A + C_SUM * Tt + C_CORR * TC) + 0x1p-40 * (A + Tt));
}

// Position of ion j as seen by move k of the current group (all earlier
// moves of the group decided).
__device__ __forceinline__ float4 position_for(const Smem &sm, const ChainDev &ch, int k0, int nk, int k, int j)
{
    const int l = j - k0;
    if (l >= 0 && l < nk) {
        if (l < k && bit(sm.accw, l)) return sm.trial[l];
        return sm.own[l];
    }
    return __ldcg(&ch.pos[j]);
}

// FP64 recomputation of move k in the oracle's arithmetic: terms in FP64 with
// IEEE sqrt and division, summed sequentially within 1024-index chunks, the
// chunk sums added in order; overlap from the FP64 squared distance.
__device__ void fp64_decide(Smem &sm, const ChainDev &ch, int k0, int nk, int k)
{
    const int tid = threadIdx.x;
    const int N = ch.N;
    const int i = k0 + k;
    const float4 a = sm.trial[k], b = sm.own[k];
    if (tid == 0) sm.ovl_flag = 0;
    double total = 0.0;
    for (int c0 = 0; c0 < N; c0 += CHUNK) {
        __syncthreads();
        for (int jj = tid; jj < CHUNK; jj += T) {
            const int j = c0 + jj;
            double t = 0.0;
            if (j < N && j != i) {
                bool o;
                t = term_fp64(a, b, position_for(sm, ch, k0, nk, k, j), o, ch.sig2);
                if (o) sm.ovl_flag = 1;
            }
            sm.chunk[jj] = t;
        }
        __syncthreads();
        if (tid == 0) {
            const int len = min(CHUNK, N - c0);
            double s = 0.0;
            for (int jj = 0; jj < len; ++jj)
                if (c0 + jj != i) s = __dadd_rn(s, sm.chunk[jj]);
            total = __dadd_rn(total, s);
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double dE = __dmul_rn(__dmul_rn(ch.lB, (double)a.w), total);
        int out;
        if (sm.ovl_flag) out = OUT_OVERLAP;
        else if (sm.st[k] & ST_UZERO) out = OUT_ACCEPT;
        else out = (dE < sm.Lneg[k]) ? OUT_ACCEPT : OUT_METROPOLIS;
        sm.outcome[k] = (signed char)out;
        sm.tier[k] = 4;
        sm.dE[k] = sm.ovl_flag ? __longlong_as_double(0x7ff8000000000000ll) : dE;
        sm.decw[k >> 5] |= 1u << (k & 31);
        if (out == OUT_ACCEPT) sm.accw[k >> 5] |= 1u << (k & 31);
    }
    __syncthreads();
}

__device__ __forceinline__ float4 pad_point(float v)
{
    return make_float4(v, v, v, 0.0f);
}

// One work item: the S moves of group g of chain `tk.chain` at sweep s.
__device__ bool process_group(Smem &sm, const ChainDev *__restrict__ chains, const Ticket tk, int ticket, Ctl *ctl)
{
    const int tid = threadIdx.x;
    const ChainDev &ch = chains[tk.chain];
    const int N = ch.N, B = ch.B, g = tk.g, k0 = g * S, nk = min(S, N - k0);
    const unsigned long long s = *ch.sweep + (unsigned long long)tk.s_rel;
    const unsigned need_prev = (unsigned)s;        // tag of a version written in sweep s-1
    const unsigned need_cur = (unsigned)(s + 1);   // tag of a version written in sweep s
    const float lo2 = ch.sig2_lo, hi2 = ch.sig2_hi;  // FP32 overlap band [lo2, hi2]
    const double sig2 = ch.sig2;
    const int mode = ctl->guard_mode;

    // 1. our group's positions after its previous move (Algorithm 1's loads)
    if (tid == 0) sm.ok = wait_group(ch, g, need_prev, ctl);
    __syncthreads();
    if (!sm.ok) return false;
    if (tid < S) {
        const int k = tid;
        unsigned stv = 0;
        if (k < nk) {
            const float4 x = __ldcg(&ch.pos[k0 + k]);
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
                sm.Lneg[k] = __longlong_as_double(0x7ff0000000000000ll);
            } else {
                sm.Lneg[k] = -series_log((double)ua * 0x1p-24);
            }
        } else {
            sm.own[k] = pad_point(-1.0e6f);
            sm.trial[k] = pad_point(-1.0e6f);
            sm.Lneg[k] = 0.0;
            stv = ST_INACTIVE;
        }
        sm.st[k] = (unsigned char)stv;
        sm.outcome[k] = -1;
        sm.tier[k] = 0;
        sm.dE[k] = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
        for (int w = 0; w < WORDS; ++w) {
            sm.ovo[k][w] = 0u;
            sm.ovn[k][w] = 0u;
        }
    }
    if (tid < WORDS) {
        sm.accw[tid] = 0u;
        sm.decw[tid] = 0u;
    }
    __syncthreads();

    // 2. pair sums: thread (p, r) owns moves p and p + S/2, column slice r
    const int p = tid / ETA, r = tid % ETA;
    const int kA = p, kB = p + S / 2;
    const float4 aA = sm.trial[kA], bA = sm.own[kA], aB = sm.trial[kB], bB = sm.own[kB];
    float sA = 0.f, sB = 0.f, AA = 0.f, AB = 0.f, TA = 0.f, TB = 0.f, CA = 0.f, CB = 0.f;
    float mA = __int_as_float(0x7f800000), mB = __int_as_float(0x7f800000);
    double SA = 0.0, SB = 0.0;

    // 2a. in-group block (Algorithms 3 and 4): upper triangle final, lower triangle both ways
    for (int j = r; j < nk; j += ETA) {
        const float4 yo = sm.own[j], yn = sm.trial[j];
        if (kA < nk) ingroup_pair(sm, kA, j, aA, bA, yo, yn, sA, AA, TA, CA, mA, lo2, hi2, sig2);
        if (kB < nk) ingroup_pair(sm, kB, j, aB, bB, yo, yn, sB, AB, TB, CB, mB, lo2, hi2, sig2);
    }
    SA += (double)sA;
    SB += (double)sB;
    sA = sB = 0.f;

    // 2b. every other group, oldest published version first (Algorithm 2 per guest group, Algorithm 5's order)
    for (int step = 1; step < B; ++step) {
        const int J = (g + step) % B;
        const unsigned need = (J > g) ? need_prev : need_cur;
        if (tid == 0) sm.ok = wait_group(ch, J, need, ctl);
        __syncthreads();
        if (!sm.ok) return false;
        if (tid < S) {
            const int idx = J * S + tid;
            sm.tile[tid] = (idx < N) ? __ldcg(&ch.pos[idx]) : pad_point(1.0e6f);
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < S / ETA; ++jj) {
            const float4 y = sm.tile[jj * ETA + r];
            pair_acc(aA, bA, y, sA, AA, TA, mA);
            pair_acc(aB, bB, y, sB, AB, TB, mB);
        }
        SA += (double)sA;
        SB += (double)sB;
        sA = sB = 0.f;
        __syncthreads();
    }

    // 2c. combine the ETA column slices
#pragma unroll
    for (int o = 1; o < ETA; o <<= 1) {
        SA += __shfl_xor_sync(FULL, SA, o);
        SB += __shfl_xor_sync(FULL, SB, o);
        AA += __shfl_xor_sync(FULL, AA, o);
        AB += __shfl_xor_sync(FULL, AB, o);
        TA += __shfl_xor_sync(FULL, TA, o);
        TB += __shfl_xor_sync(FULL, TB, o);
        CA += __shfl_xor_sync(FULL, CA, o);
        CB += __shfl_xor_sync(FULL, CB, o);
        mA = fminf(mA, __shfl_xor_sync(FULL, mA, o));
        mB = fminf(mB, __shfl_xor_sync(FULL, mB, o));
    }
    if (r == 0) {
        // FP32 accumulations of the bound quantities are inflated by 2^-10 (>= their own rounding error)
        sm.base[kA] = SA;
        sm.Ab[kA] = AA * (1.0f + 0x1p-10f);
        sm.Tb[kA] = TA * (1.0f + 0x1p-10f);
        sm.TCb[kA] = CA * (1.0f + 0x1p-10f);
        sm.mind2[kA] = mA;
        sm.base[kB] = SB;
        sm.Ab[kB] = AB * (1.0f + 0x1p-10f);
        sm.Tb[kB] = TB * (1.0f + 0x1p-10f);
        sm.TCb[kB] = CB * (1.0f + 0x1p-10f);
        sm.mind2[kB] = mB;
    }
    __syncthreads();

    // 3. decisions.  3a: moves decided without any in-group dependence.
    if (tid < S) {
        const int k = tid;
        unsigned stv = sm.st[k];
        bool dec = false;
        if (stv & ST_INACTIVE) {
            dec = true;
        } else if (stv & ST_WALL) {
            dec = true;
            sm.outcome[k] = OUT_WALL;
        } else {
            const float m2 = sm.mind2[k];
            if (m2 < lo2) stv |= ST_OVL_CERTAIN;
            else if (!(m2 > hi2)) stv |= ST_OVL_AMBIG;  // inside the band (or NaN): FP64 decides
            sm.st[k] = (unsigned char)stv;
            if (stv & ST_OVL_CERTAIN) {
                dec = true;
                sm.outcome[k] = OUT_OVERLAP;
            }
        }
        const unsigned bal = __ballot_sync(FULL, dec);
        if ((tid & 31) == 0) sm.decw[tid >> 5] = bal;
    }
    __syncthreads();

    // 3b: moves whose outcome is the same for every combination of the
    // undecided earlier outcomes of the group (interval over the corrections).
    if (tid < S) {
        const int k = tid;
        bool dec = bit(sm.decw, k);
        if (!dec && !(sm.st[k] & ST_OVL_AMBIG)) {
            float lo = 0.f, hi = 0.f;
            bool ovl_c = false, ovl_p = false;
            for (int j = 0; j < k; ++j) {
                if (bit(sm.decw, j)) {  // decided so far means rejected: old position
                    ovl_c |= bit(sm.ovo[k], j);
                } else {
                    const float c = sm.cmat[j * CS + k];
                    lo += fminf(c, 0.f);
                    hi += fmaxf(c, 0.f);
                    const bool bo = bit(sm.ovo[k], j), bn = bit(sm.ovn[k], j);
                    if (bo && bn) ovl_c = true;
                    else if (bo || bn) ovl_p = true;
                }
            }
            if (ovl_c) {
                dec = true;
                sm.outcome[k] = OUT_OVERLAP;
            } else if (!ovl_p) {
                if (sm.st[k] & ST_UZERO) {
                    dec = true;
                    sm.outcome[k] = OUT_ACCEPT;
                } else if (mode != 1) {
                    const double lq = __dmul_rn(ch.lB, (double)sm.own[k].w);
                    const double e1 = lq * (sm.base[k] + (double)lo), e2 = lq * (sm.base[k] + (double)hi);
                    const double bnd = band(sm, k, fabs(lq), mode) + 0x1p-50 * (fabs(e1) + fabs(e2) + fabs(sm.Lneg[k]));
                    if (isfinite(e1) && isfinite(e2)) {
                        const double elo = e1 < e2 ? e1 : e2, ehi = e1 < e2 ? e2 : e1;
                        if (ehi < sm.Lneg[k] - bnd) {
                            dec = true;
                            sm.outcome[k] = OUT_ACCEPT;
                        } else if (elo > sm.Lneg[k] + bnd) {
                            dec = true;
                            sm.outcome[k] = OUT_METROPOLIS;
                        }
                    }
                }
            }
        }
        const unsigned bal = __ballot_sync(FULL, dec);
        const unsigned acc = __ballot_sync(FULL, dec && sm.outcome[k] == OUT_ACCEPT);
        if ((tid & 31) == 0) {
            sm.decw[tid >> 5] = bal;
            sm.accw[tid >> 5] = acc;
        }
    }
    __syncthreads();
    // moves settled in 3b (not rejected by wall/overlap before any dependence) are "interval" decisions
    // 3c: the rest in order, one warp, exact sums; FP64 for moves inside the band.
    for (;;) {
        if (tid < 32) {
            const int lane = tid;
            int k = 0;
            int guard = -1;
            for (;;) {
                // next undecided move
                int nxt = -1;
#pragma unroll
                for (int w = 0; w < WORDS; ++w) {
                    const unsigned und = ~sm.decw[w];
                    if (nxt < 0 && und) nxt = w * 32 + __ffs(und) - 1;
                }
                if (nxt < 0 || nxt >= nk) break;
                k = nxt;
                float part = 0.f;
                for (int j = lane; j < k; j += 32)
                    if (bit(sm.accw, j)) part += sm.cmat[j * CS + k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
                if (lane == 0) {
                    bool ovl = false;
#pragma unroll
                    for (int w = 0; w < WORDS; ++w) {
                        const unsigned below = (w * 32 + 32 <= k) ? FULL : (w * 32 >= k ? 0u : ((1u << (k - w * 32)) - 1u));
                        ovl |= ((sm.ovn[k][w] & sm.accw[w]) | (sm.ovo[k][w] & ~sm.accw[w])) & below;
                    }
                    int out = -1;
                    double dE = __longlong_as_double(0x7ff8000000000000ll);
                    if (ovl) {
                        out = OUT_OVERLAP;
                    } else if (sm.st[k] & ST_OVL_AMBIG) {
                        out = -2;  // exact overlap needs FP64
                    } else {
                        const double lq = __dmul_rn(ch.lB, (double)sm.own[k].w);
                        dE = lq * (sm.base[k] + (double)part);
                        if (sm.st[k] & ST_UZERO) {
                            out = OUT_ACCEPT;
                        } else {
                            const double bnd = band(sm, k, fabs(lq), mode) + 0x1p-50 * (fabs(dE) + fabs(sm.Lneg[k]));
                            if (dE < sm.Lneg[k] - bnd) out = OUT_ACCEPT;
                            else if (dE > sm.Lneg[k] + bnd) out = OUT_METROPOLIS;
                            else out = -2;
                        }
                    }
                    if (out == -2) {
                        guard = k;
                    } else {
                        sm.outcome[k] = (signed char)out;
                        sm.tier[k] = 1;
                        sm.dE[k] = dE;
                        sm.decw[k >> 5] |= 1u << (k & 31);
                        if (out == OUT_ACCEPT) sm.accw[k >> 5] |= 1u << (k & 31);
                    }
                }
                guard = __shfl_sync(FULL, guard, 0);
                __syncwarp();
                if (guard >= 0) break;
            }
            if (lane == 0) sm.guard_k = guard;
        }
        __syncthreads();
        const int gk = sm.guard_k;
        if (gk < 0) break;
        fp64_decide(sm, ch, k0, nk, gk);
    }

    // 4. publish: final positions, then the sweep-tagged words with the accept bits
    if (tid < nk) {
        const bool acc = bit(sm.accw, tid);
        __stcg(&ch.pos[k0 + tid], acc ? sm.trial[tid] : sm.own[tid]);
    }
    __syncthreads();
    const bool publish = (long long)ticket != ctl->skip_ticket;
    if (tid == 0 && publish) {
        __threadfence();
        const int nw = (nk + 31) / 32;
        for (int w = 0; w < nw; ++w)
            st_release(&ch.flags[g * WORDS + w], ((unsigned long long)need_cur << 32) | sm.accw[w]);
    }

    // 5. bookkeeping off the critical path: dE of moves decided by interval, ledger, counters, records
    double mydE = 0.0;
    if (tid < nk) {
        const int k = tid;
        const int out = sm.outcome[k];
        const bool need_sum = (out == OUT_ACCEPT || out == OUT_METROPOLIS) && sm.tier[k] == 0 &&
                              !(sm.st[k] & ST_UZERO);
        const bool acc_uzero = (out == OUT_ACCEPT) && sm.tier[k] == 0 && (sm.st[k] & ST_UZERO);
        if (need_sum || acc_uzero || (ch.rec && out != OUT_WALL && out != OUT_OVERLAP && sm.tier[k] != 4)) {
            float part = 0.f;
            for (int j = 0; j < k; ++j)
                if (bit(sm.accw, j)) part += sm.cmat[j * CS + k];
            const double lq = __dmul_rn(ch.lB, (double)sm.own[k].w);
            if (sm.tier[k] == 0) sm.dE[k] = lq * (sm.base[k] + (double)part);
        }
        if (out == OUT_ACCEPT) mydE = sm.dE[k];
    }
    // deterministic block sum of the accepted dE (fixed tree order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mydE += __shfl_xor_sync(FULL, mydE, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = mydE;
    __syncthreads();
    if (tid == 0 && publish) {
        double gsum = 0.0;
        for (int w = 0; w < T / 32; ++w) gsum += sm.red[w];
        // fold into the chain ledger in stream order
        const unsigned long long me = s * (unsigned long long)B + (unsigned long long)g;
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        bool ok = true;
        while (ld_acquire(ch.ledger_seq) != me) {
            if (*(volatile int *)&ctl->abort) {
                ok = false;
                break;
            }
            if (++spins > 32) __nanosleep(40);
            if ((spins & 63) == 0 && (long long)(globaltimer() - t0) > ctl->timeout_ns) {
                atomicCAS(&ctl->err, 0, KERR_TIMEOUT);
                atomicExch(&ctl->abort, 1);
                ok = false;
                break;
            }
        }
        if (ok) {
            volatile double *L = ch.ledger;
            *L = *L + gsum;
            st_release(ch.ledger_seq, me + 1);
        }
        sm.ok = ok ? 1 : 0;
    }
    if (tid < 32) {
        // counters by outcome
        unsigned cnt[6] = {0, 0, 0, 0, 0, 0};
        for (int k = tid; k < nk; k += 32) {
            const int out = sm.outcome[k];
            if (out >= 0 && out <= 3) cnt[out]++;
            if (sm.tier[k] == 4) cnt[4]++;
            if (sm.tier[k] == 0 && (out == OUT_ACCEPT || out == OUT_METROPOLIS)) cnt[5]++;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt[c] += __shfl_xor_sync(FULL, cnt[c], o);
        }
        if (tid == 0) {
            atomicAdd(&ch.stats[CNT_ACCEPT], (unsigned long long)cnt[OUT_ACCEPT]);
            atomicAdd(&ch.stats[CNT_METRO], (unsigned long long)cnt[OUT_METROPOLIS]);
            atomicAdd(&ch.stats[CNT_OVERLAP], (unsigned long long)cnt[OUT_OVERLAP]);
            atomicAdd(&ch.stats[CNT_WALL], (unsigned long long)cnt[OUT_WALL]);
            atomicAdd(&ch.stats[CNT_FP64], (unsigned long long)cnt[4]);
            atomicAdd(&ch.stats[CNT_INTERVAL], (unsigned long long)cnt[5]);
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
            const double lq = __dmul_rn(ch.lB, (double)sm.own[k].w);
            rc.scale = fabs(lq) * (double)sm.Ab[k];
            const int out = sm.outcome[k];
            rc.dE = (out == OUT_ACCEPT || out == OUT_METROPOLIS) ? sm.dE[k] : __longlong_as_double(0x7ff8000000000000ll);
            double d32 = __longlong_as_double(0x7ff8000000000000ll);
            if (out == OUT_ACCEPT || out == OUT_METROPOLIS) {
                float part = 0.f;
                for (int j = 0; j < k; ++j)
                    if (bit(sm.accw, j)) part += sm.cmat[j * CS + k];
                d32 = lq * (sm.base[k] + (double)part);
            }
            rc.dE32 = d32;
            ch.rec[idx] = rc;
        }
    }
    __syncthreads();
    return sm.ok != 0;
}

__global__ void __launch_bounds__(T, 2)
sweep_kernel(const ChainDev *__restrict__ chains, const Ticket *__restrict__ sched, int n_tickets, Ctl *ctl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&ctl->ticket, 1u);
            const int ab = *(volatile int *)&ctl->abort;
            sm.ticket = (ab || t >= (unsigned)n_tickets) ? -1 : (int)t;
        }
        __syncthreads();
        const int t = sm.ticket;
        __syncthreads();
        if (t < 0) return;
        if (!process_group(sm, chains, sched[t], t, ctl)) return;
    }
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
    return cudaFuncSetAttribute(mcg::sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(mcg::Smem));
}

cudaError_t sweep_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcg::sweep_kernel, mcg::T, sizeof(mcg::Smem));
}

cudaError_t sweep_launch(int grid, const mcg::ChainDev *chains, const mcg::Ticket *sched, int n_tickets, mcg::Ctl *ctl,
                         int n_chains, long long n_sweeps, cudaStream_t st)
{
    mcg::sweep_kernel<<<grid, mcg::T, sizeof(mcg::Smem), st>>>(chains, sched, n_tickets, ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mcg::advance_sweeps<<<(n_chains + 127) / 128, 128, 0, st>>>(chains, n_chains, n_sweeps, ctl);
    return cudaGetLastError();
}

}  // namespace mcg_host
