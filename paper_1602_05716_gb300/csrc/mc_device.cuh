// mc_device.cuh -- device building blocks of the sm_103a sequential-Metropolis
// path: the Philox4x32-10 stream, the FP64 logarithm of the acceptance test,
// the FP64 canonical pair term, and the structures shared by the kernels and
// the host runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcg {

// ---------------------------------------------------------------------------
// Work decomposition.  A "group" is S consecutive ions of one chain; a work
// item ("ticket") is one group at one sweep.  A CTA of T threads owns the S
// trial moves of its group.
constexpr int S = 128;          // moves per group
constexpr int T = 256;          // threads per CTA
constexpr int ETA = T / (S / 2);  // threads per pair of moves (column slices)
constexpr int CS = S + 8;       // row stride of the correction matrix (floats)
constexpr int CHUNK = 1024;     // canonical FP64 summation chunk
constexpr int WORDS = S / 32;   // 32-move flag words per group

// Outcome codes (same meaning as the records of the C ABI).
constexpr int OUT_ACCEPT = 0;
constexpr int OUT_METROPOLIS = 1;
constexpr int OUT_OVERLAP = 2;
constexpr int OUT_WALL = 3;

// Error codes written by the kernel into Ctl::err.
constexpr int KERR_TIMEOUT = 1;
constexpr int KERR_PROTOCOL = 2;

struct MoveRec {
    unsigned long long m;
    int i;
    int outcome;
    double dE;
    double dE32;
    double bound;  // proven FP32 error bound of dE32 (static part), +inf when the band was disabled
    double dEt;    // surrogate energy change of a delayed-acceptance move (NaN otherwise)
    int tier;
    int pad;
};

// Per-work-item timeline (mc_trace_enable): %globaltimer nanoseconds.
struct TraceRec {
    unsigned long long item;   // absolute stream index sweep * B + group
    unsigned long long t_start, t_ready, t_window, t_resolved, t_published;
    unsigned long long n_guard;
    unsigned long long t_positions;
    unsigned long long t_tile, t_tiles, t_w2;  // last tile observed, tiles done, second window observed
    unsigned long long t_ph[4];                // slices combined, band ready, round 0 done, oldest deep window observed
    unsigned int c_res[8];                     // SM cycles from the window's outcome to the resolve checkpoints
};

// Per-chain device descriptor (read-only during a launch).
struct DADev;

struct ChainDev {
    float4 *pos[2];               // 2 x N_pad entries: x, y, z, valence (Sec. 3.1's float4 layout); the
                                  // positions after sweep v live in pos[(v + 1) & 1]
    unsigned long long *flags;    // per 32-ion word: ((sweep+1) << 32) | accept bits, released after the positions
    unsigned long long *bits;     // per 32-ion word: the same value, stored as soon as the outcomes are known
    double *ledger;               // running energy
    unsigned long long *ledger_seq;  // groups folded into the ledger (absolute stream index)
    unsigned long long *stats;    // 8 counters
    unsigned long long *sweep;    // completed sweeps (absolute)
    unsigned long long sweep_base;  // sweep count when the positions were last set from the host
    MoveRec *rec;                 // validation records or nullptr
    TraceRec *trace;              // work-item timeline or nullptr
    long long trace_cap;
    unsigned long long rec_sweep0;  // sweep at which recording started
    long long rec_cap;
    double *eser;                 // energy series: the ledger after each sweep (mc_energy_series_enable) or nullptr
    long long eser_cap;
    unsigned long long eser_sweep0;  // sweep stored in eser[0]
    int N;
    int B;                        // groups: ceil(N / S)
    float D;                      // fl32(2h)
    float sig2_lo;                // FP32 squared distances below this certainly overlap
    float sig2_hi;                // ... above this certainly do not; in between FP64 decides
    float a_max;                  // 2 sum_j |q_j| / sigma: bounds sum_j |q_j| (1/r' + 1/r) of a valid move
    double sig2;                  // sigma^2
    double lB;                    // Bjerrum length
    double Rc2;                   // (R - sigma/2)^2
    unsigned key0, key1, ctr3;    // Philox key (seed_lo, chain_id), counter word 3 (seed_hi)
    unsigned pf;                  // 1: da is an overlap prefilter (the plain chain's decisions), 0 otherwise
    const struct DADev *da;       // delayed-acceptance state, nullptr for the plain chain
};

struct Ticket {
    int chain;
    int g;
    int s_rel;
    int pad;
};

struct Ctl {
    unsigned int ticket;          // next work item
    int err;                      // KERR_*
    int abort;                    // set on any error: every CTA leaves
    int guard_mode;               // 0 band, 1 always FP64, 2 never, 3 always through the tiers
    long long timeout_ns;
    long long skip_ticket;        // fault injection (-1 off)
    unsigned long long err_info;  // where a wait gave up
    int pairs;                    // 1: clusters of two CTAs share each work item's tiles (leader even, helper odd)
    int deep;                     // 1: deep windows (groups g-2.. both ways, corrections in tensor memory)
    struct PairBox *box;          // per cluster: the work item and the helper's per-move tile sums
    // shared guard: a work item whose move needs an accurate recomputation posts it on the board, and every warp
    // that waits in wait_words takes chunks of its pair sum
    struct GuardBoard *gb;        // nullptr: every guard tier runs on its own work item's CTA
    unsigned long long gnext;     // (request id << 32) | (chunks << 16) | next chunk to take
    unsigned gdone;               // chunks of the current request finished
    unsigned glock;               // 1 while a work item holds the board
};

// The posted guard request: the move (ion i of group g, old position b, trial a), where its partners' positions
// are published, and the groups whose positions it sees from its work item's shared memory (GB_SLOTS of them:
// its own group, the window, the deep windows; group -1 for an unused slot).  part / bpart: per chunk of
// GB_CHUNK ions, the sum of the pair terms and of their error bounds.
constexpr int GB_CHUNK = 4096, GB_SLOTS = 5;
struct GuardBoard {
    int tier, N, g, i;
    float dn, rho0;               // tier 2: bound of the move's length, smallest partner distance to [b, a]
    int pad0[2];
    float4 a, b;
    const float4 *Pprev, *Pcur;
    int slotJ[GB_SLOTS];
    int pad[3];
    float4 ovl[GB_SLOTS][128];
    double *part, *bpart;
};

// Hand-over from a cluster's helper CTA to its leader (global memory, ordered by the cluster barriers).
struct PairBox {
    int ticket;
    int pad[3];
    float h[128], l[128], p[128], m[128];  // per move: float-float tile sum, P sum, minimum squared distance
};

// Counter slots of ChainDev::stats.
constexpr int CNT_ACCEPT = 0, CNT_METRO = 1, CNT_OVERLAP = 2, CNT_WALL = 3, CNT_FP64 = 4, CNT_INTERVAL = 5,
              CNT_T2 = 6, CNT_T3 = 7, CNT_T4 = 8, CNT_ROUNDS = 9, CNT_CYC_WIN = 10, CNT_CYC_TILES = 11,
              CNT_CYC_RESOLVE = 12, CNT_CYC_GUARD = 13, CNT_CYC_TOTAL = 14, CNT_CYC_T2 = 15, CNT_CYC_T3 = 16,
              CNT_CYC_T4 = 17, CNT_OVL_SCAN = 18, CNT_CYC_OVL = 19, CNT_DA_REJ1 = 20, CNT_DA_OVL1 = 21,
              CNT_DA_FP64 = 22, CNT_CYC_DA1 = 23, CNT_CYC_DA_PART = 24;  // 24..27: grid, features, MLP, near field
constexpr int NCOUNTERS = 32;
constexpr float U32 = 0x1p-24f;  // unit roundoff of FP32

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): two 32x32 multiplies per round with
// the published multipliers; key bumped by the published Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Draws of move m: counter (m_lo, m_hi, purpose, seed_hi), key (seed_lo, chain).
__device__ __forceinline__ uint4 move_draws(const ChainDev &ch, unsigned long long m, unsigned purpose)
{
    return philox4x32_10(make_uint4((unsigned)m, (unsigned)(m >> 32), purpose, ch.ctr3), make_uint2(ch.key0, ch.key1));
}

// Trial position: x'_k = fl32(x_k + fl32((u_k - 1/2) D)), u_k = (w_k >> 8) 2^-24
// (Algorithm 1: displacement (u - 0.5) D added to the old coordinate).
__device__ __forceinline__ float trial_coord(float x, unsigned w, float D)
{
    const float u = __uint2float_rn(w >> 8) * 0x1p-24f;
    return __fadd_rn(x, __fmul_rn(__fsub_rn(u, 0.5f), D));
}

// ---------------------------------------------------------------------------
// L(u): natural logarithm in FP64 from IEEE +, -, *, / only, so that every
// implementation of the same steps returns the same double.  Reduction
// u = f 2^e with f in [sqrt(1/2), sqrt(2)); ln f = 2 atanh(s) with
// s = (f - 1)/(f + 1) summed as 2 s (1 + z/3 + ... + z^10/21), z = s^2
// (Abramowitz & Stegun 4.1.27); ln 2 split into a 32-bit head and a tail.
__device__ __forceinline__ double series_log(double u)
{
    int e;
    double f = frexp(u, &e);
    if (f < 0.70710678118654752440) {
        f = __dmul_rn(f, 2.0);
        e -= 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double z = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, 21.0);
#pragma unroll
    for (int k = 9; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, z), __ddiv_rn(1.0, (double)(2 * k + 1)));
    const double lnf = __dmul_rn(__dmul_rn(2.0, s), p);
    const double de = (double)e;
    return __dadd_rn(__dmul_rn(de, 0.693147180601954460144042968750),
                     __dadd_rn(__dmul_rn(de, -4.2009150726810847291823431924e-11), lnf));
}

// FP64 squared distance of two FP32 points, in the order ((dx^2 + dy^2) + dz^2).
__device__ __forceinline__ double d2_fp64(float ax, float ay, float az, float bx, float by, float bz)
{
    const double dx = __dsub_rn((double)ax, (double)bx);
    const double dy = __dsub_rn((double)ay, (double)by);
    const double dz = __dsub_rn((double)az, (double)bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// FP64 pair term q_j (1/|a - y| - 1/|b - y|) with IEEE sqrt and division.
__device__ __forceinline__ double term_fp64(float4 a, float4 b, float4 y, bool &ovl, double sig2)
{
    const double d2n = d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z);
    const double d2o = d2_fp64(b.x, b.y, b.z, y.x, y.y, y.z);
    ovl = d2n < sig2;
    const double rn = __ddiv_rn(1.0, __dsqrt_rn(d2n));
    const double ro = __ddiv_rn(1.0, __dsqrt_rn(d2o));
    return __dmul_rn((double)y.w, __dsub_rn(rn, ro));
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Release / acquire accesses at GPU scope for the inter-CTA protocol.
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Flush-to-zero forms for the pair loop: the same accuracy on normal inputs
// (inverse distances of ions at least sigma apart inside a finite sphere).
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_ftz(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Accurate FP32 pair term of move (old b, displacement d = a - b) against an ion y whose position is
// settled for this move (every other group's tile, and the later ions of this group).  With e = y - b,
// q_y (1/|a-y| - 1/|b-y|) = q_y Dd (rn ro)^2 / (rn + ro) where Dd = d . (2e - d) = |b-y|^2 - |a-y|^2: no
// difference of two nearly equal inverse distances, so the rounding error scales with |d| / r^2 instead
// of 1/r and the FP32 band stays narrow at large N.  Accumulates the term into s, |term| into Tt,
// |q_y| rn ro into P (the bound's second sum) and the trial's squared distance into the minimum mn.
__device__ __forceinline__ void pair_far(const float3 b, const float3 d, const float4 y, float &s, float &Tt, float &P,
                                         float &mn)
{
    const float ex = y.x - b.x, ey = y.y - b.y, ez = y.z - b.z;
    const float Do = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
    const float wx = fmaf(2.0f, ex, -d.x), wy = fmaf(2.0f, ey, -d.y), wz = fmaf(2.0f, ez, -d.z);
    const float Dd = fmaf(d.z, wz, fmaf(d.y, wy, d.x * wx));
    const float Dn = Do - Dd;
    const float ro = rsqrt_ftz(Do), rn = rsqrt_ftz(Dn);
    const float pr = rn * ro;
    const float t = (Dd * pr) * (pr * rcp_ftz(rn + ro));
    s = fmaf(y.w, t, s);
    Tt = fmaf(fabsf(y.w), fabsf(t), Tt);
    P = fmaf(fabsf(y.w), pr, P);
    mn = fminf(mn, Dn);
}

// Packed FP32 pairs (sm_100 family): each lane of add/sub/mul/fma .f32x2 is the IEEE round-to-nearest result of
// the scalar operation, so packed code gives bit-identical values at half the issue slots.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void upk2(f32x2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Two moves (packed old positions b, doubled displacements t = 2d and m = -|d|^2) against one settled ion y.  With
// e = y - b:
//   Do = |e|^2,   Dd = 2 d.e - |d|^2 = |b - y|^2 - |a - y|^2 (three FMAs on m),   Dn = Do - Dd,
// then the term with two MUFU operations:
//   s = rsqrt(Do Dn) = rn ro,   w = rsqrt(Do + Dn + 2 (Do Dn) s) = 1 / (sqrt(Do) + sqrt(Dn)) = rn ro / (rn + ro),
//   t = (Dd s) w = Dd (rn ro)^2 / (rn + ro).
// Dd's rounding: m = -fl(|d|^2) is within 3u |d|^2 and the FMA chain adds 3u (2 |d.e|_1 + |d|^2), so Dd is within
// 6u dn (Ro + dn) of 2 d.e' - |d|^2 for the rounded e' (e's own rounding is the perturbation term of the bound, as
// for pair_far's form).  Relative error of t beyond Dd's own: with Do, Dn off by delta_o, delta_n (relative), s is
// within (|delta_o| + |delta_n| + u) / 2 + 2^-22.9, sqrt(Do Dn) = (Do Dn) s within that + u, Do + Dn + 2 sqrt(Do Dn)
// (a sum of positive terms) within max(|delta_o|, |delta_n|) + 4.7u, w within half of that + 2^-22.9, so t is within
// |delta_o| + |delta_n| + 9.2u: below the rel(Dn) + 19u (|delta_o| <= 3u) of the per-term bound far_coeffs uses.
// Without the |t| sum (|t| <= dn rn ro exactly, so the bound takes dn P); P sums |q| s, which is within
// rel(Dn) / 2 + 5u of rn ro, inside the bound's 2^-16 slack for the rounding of rn ro.
struct Mv2 {
    f32x2 bx, by, bz, tx, ty, tz, m;
};

__device__ __forceinline__ void pair_far2(const Mv2 &m, const float4 y, f32x2 &s, f32x2 &P, float &mn0, float &mn1)
{
    const f32x2 two = pk2(2.0f, 2.0f);
    const f32x2 ex = sub2(pk2(y.x, y.x), m.bx), ey = sub2(pk2(y.y, y.y), m.by), ez = sub2(pk2(y.z, y.z), m.bz);
    const f32x2 Do = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
    const f32x2 Dd = fma2(m.tz, ez, fma2(m.ty, ey, fma2(m.tx, ex, m.m)));
    const f32x2 Dn = sub2(Do, Dd);
    const f32x2 pd = mul2(Do, Dn);
    float p0, p1;
    upk2(pd, p0, p1);
    const f32x2 sr = pk2(rsqrt_ftz(p0), rsqrt_ftz(p1));
    const f32x2 c2 = fma2(two, mul2(pd, sr), add2(Do, Dn));
    float c0, c1;
    upk2(c2, c0, c1);
    const f32x2 w = pk2(rsqrt_ftz(c0), rsqrt_ftz(c1));
    const f32x2 t = mul2(mul2(Dd, sr), w);
    s = fma2(pk2(y.w, y.w), t, s);
    P = fma2(pk2(fabsf(y.w), fabsf(y.w)), sr, P);
    float Dn0, Dn1;
    upk2(Dn, Dn0, Dn1);
    mn0 = fminf(mn0, Dn0);
    mn1 = fminf(mn1, Dn1);
}

// One move against one settled ion: lane 0 of pair_far2's arithmetic, operation for operation (every packed lane
// rounds like the scalar operation), for a third occupied layer of 32 move slots.
__device__ __forceinline__ void pair_far1(const Mv2 &m, const float4 y, float &s, float &P, float &mn)
{
    float bx, by, bz, tx, ty, tz, mm, u;
    upk2(m.bx, bx, u);
    upk2(m.by, by, u);
    upk2(m.bz, bz, u);
    upk2(m.tx, tx, u);
    upk2(m.ty, ty, u);
    upk2(m.tz, tz, u);
    upk2(m.m, mm, u);
    const float ex = __fsub_rn(y.x, bx), ey = __fsub_rn(y.y, by), ez = __fsub_rn(y.z, bz);
    const float Do = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
    const float Dd = __fmaf_rn(tz, ez, __fmaf_rn(ty, ey, __fmaf_rn(tx, ex, mm)));
    const float Dn = __fsub_rn(Do, Dd);
    const float pd = __fmul_rn(Do, Dn);
    const float sr = rsqrt_ftz(pd);
    const float c2 = __fmaf_rn(2.0f, __fmul_rn(pd, sr), __fadd_rn(Do, Dn));
    const float w = rsqrt_ftz(c2);
    const float t = __fmul_rn(__fmul_rn(Dd, sr), w);
    s = __fmaf_rn(y.w, t, s);
    P = __fmaf_rn(fabsf(y.w), sr, P);
    mn = fminf(mn, Dn);
}

// The packed move data of two moves (old positions b0, b1; displacements d0, d1 as FP32 differences a - b).
__device__ __forceinline__ Mv2 make_mv2(const float3 b0, const float3 d0, const float3 b1, const float3 d1)
{
    Mv2 v;
    v.bx = pk2(b0.x, b1.x);
    v.by = pk2(b0.y, b1.y);
    v.bz = pk2(b0.z, b1.z);
    v.tx = pk2(2.0f * d0.x, 2.0f * d1.x);
    v.ty = pk2(2.0f * d0.y, 2.0f * d1.y);
    v.tz = pk2(2.0f * d0.z, 2.0f * d1.z);
    v.m = pk2(-__fmaf_rn(d0.z, d0.z, __fmaf_rn(d0.y, d0.y, __fmul_rn(d0.x, d0.x))),
              -__fmaf_rn(d1.z, d1.z, __fmaf_rn(d1.y, d1.y, __fmul_rn(d1.x, d1.x))));
    return v;
}

// Asynchronous 16-byte copy global -> shared through L2 (cp.async.cg); cp_async_wait_all waits for all of this
// thread's copies.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Error-free transformations in FP32 (Knuth's TwoSum, FMA-based TwoProduct).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace mcg
