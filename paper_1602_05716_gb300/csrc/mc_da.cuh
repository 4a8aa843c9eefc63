// mc_da.cuh -- device-side definitions of delayed acceptance (a two-stage
// Metropolis test in the sense of Christen & Fox, 2005) on top of the exact
// sequential chain of Sec. 2.
//
// Stage 1 decides on a cheap surrogate energy change
//     dEt = l_B q_i ([phi_near + g(v)](x') - [phi_near + g(v)](x)),
// phi_near the Coulomb sum over counted ions within r_c (exact up to
// r_s = r_c / 2, then a C1 taper 1 - t^2 (3 - 2t) so that an ion crossing r_c
// changes it continuously) and g a 33-64-64-1 SiLU MLP with BF16 weights fed
// with the net valence of counted ions in 32 shells (equal width in d^2) of
// the taper region around the point, and its radial coordinate.  Survivors pay the exact O(N) sum of
// the plain chain and are accepted with min(1, exp(-(dE - dEt))).
//
// Counted ions for the move of ion i in group g: every ion except i, the
// earlier ions of g and all ions of the W groups tried just before g (cyclic
// over the sweep).  The set depends only on the move index, so dEt is a
// function of the current state (the delayed-acceptance ratio then keeps the
// chain's stationary distribution exactly).  W is at least the number of
// resident CTAs plus one, so every counted ion's current position is final
// when the work item starts: stage 1 of all S moves of a group runs before
// the pair sums, which then cover the stage-1 survivors only.
#pragma once

#include "mc_device.cuh"

namespace mcg {

constexpr int DA_NIN = 33, DA_H = 64;                                           // MLP shape
constexpr int DA_NP = DA_H * DA_NIN + DA_H + DA_H * DA_H + DA_H + DA_H + 1;    // 6401 parameters
constexpr int DA_OFF_B1 = DA_H * DA_NIN, DA_OFF_W2 = DA_OFF_B1 + DA_H, DA_OFF_B2 = DA_OFF_W2 + DA_H * DA_H,
              DA_OFF_W3 = DA_OFF_B2 + DA_H, DA_OFF_B3 = DA_OFF_W3 + DA_H;
constexpr int OUT_DA1 = 4;  // outcome: rejected by the surrogate stage

// Per-chain delayed-acceptance state (device memory, written by the host at
// set-up and by the per-sweep preparation kernels).
struct DADev {
    const unsigned short *w;       // BF16 weights, layout W1[64][33], b1, W2[64][64], b2, W3, b3
    const float *w2n;              // ||W2[o]||_1, rounded up (error bound of the second layer)
    const int *cell_start;         // near-field cell list of the sweep's start positions (ncell + 1)
    const int *cell_ions;          // ion indices in cell order (N)
    float4 *cell_pos;              // their positions in cell order; accepted moves write theirs in place
    const int *slot_of;            // slot of ion j in the cell order (N)
    double rc2, rs2;               // r_c^2, r_s^2
    double rs, tw;                 // taper start r_c / 2 and width r_c - r_s
    double R;                      // sphere radius (radial input)
    float rs_f, itw_f;             // fl32(r_s), fl32(1 / width) for the FP32 taper
    float rc2_lo, rc2_hi;          // FP32 squared distances below/above certainly inside/outside r_c
    float rs2_lo, rs2_hi;          // ... below/above certainly inside/outside r_s
    float rs2_f, c32_f;            // fl32(r_s^2), fl32(32 / (r_c^2 - r_s^2)) for the FP32 shell index
    float nf_scale, nf_R;          // near-field cell of x: floor((x + nf_R) * nf_scale)
    float nf_edge;                 // its edge (>= reach / 2, so the cells within two of x's cover the reach)
    float reach2;                  // (r_c + largest trial + largest move of the candidate)^2, with slack
    float Rr;                      // fl32(R) for the FP32 radial input
    int nf_G;                      // near-field cells per axis
    int W;                         // exclusion depth in groups
    int mlp_zero;                  // every weight is +-0, so g = 0 exactly: the FP32 MLP pass is skipped
    // overlap prefilter (mc_set_overlap_prefilter): no surrogate and no stage-1 Metropolis test, stage 1 only
    // rejects trials that overlap a counted ion.  Bucket layout: cell q holds ions in slots q cap ..
    // q cap + min(cell_cnt[q], cap) - 1, each the position with the ion's index as the fourth word; an ion that
    // finds its cell full has slot_of -1 and is not listed.
    const int *cell_cnt;
    float ovl_reach2;              // (sigma + the largest move of a candidate since the sweep's start)^2, with slack
    int cap;                       // slots per cell
    int prefilter;                 // 1: the prefilter, 0: delayed acceptance
};

__device__ __forceinline__ int da_ncell_axis(const DADev &d, float x)
{
    const int c = (int)floorf((x + d.nf_R) * d.nf_scale);
    return c < 0 ? 0 : (c > d.nf_G - 1 ? d.nf_G - 1 : c);
}

__device__ __forceinline__ float bf16f(unsigned short b)
{
    return __uint_as_float((unsigned)b << 16);
}

// Is ion j counted for the move of ion i (group g = i / S) in a chain of B groups, exclusion depth Wg = min(W, B-1)?
__device__ __forceinline__ bool da_counted(int i, int g, int B, int Wg, int j)
{
    if (j == i) return false;
    const int J = j / S;
    if (J == g) return j > i;
    int back = g - J;
    if (back < 0) back += B;
    return back > Wg;
}

// exp(x) in FP64 from +, -, *, / only, the steps of the reference definition:
// x = k ln2 + r, k = round-half-even(x / ln2_head), r = (x - k ln2_head) - k ln2_tail;
// exp(r) by twenty nested Horner steps p = 1 + (p r) / m, m = 20 .. 1; scaled by 2^k.
// Zero below -700, +inf above 709.
__device__ __forceinline__ double series_exp(double x)
{
    const double head = 0.693147180601954460144042968750, tail = -4.2009150726810847291823431924e-11;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -700.0) return 0.0;
    const double kd = rint(__ddiv_rn(x, head));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, head)), __dmul_rn(kd, tail));
    double p = 1.0;
#pragma unroll 1
    for (int m = 20; m >= 1; --m) p = __dadd_rn(1.0, __ddiv_rn(__dmul_rn(p, r), (double)m));
    return scalbn(p, (int)kd);
}

// The near-field taper s(d) in FP32: 1 up to r_s, 1 - t^2 (3 - 2t) beyond.  Its error is below 22u (|s'| <= 1.5
// times the error of t, itself below 12u for d <= 2 r_s, plus four roundings).
__device__ __forceinline__ float da_taper32(const DADev &d, float dist)
{
    if (!(dist > d.rs_f)) return 1.0f;
    const float t = (dist - d.rs_f) * d.itw_f;
    return 1.0f - (t * t) * (3.0f - 2.0f * t);
}

// ... and the reference FP64 term q s(d) / d (the oracle's operations in its order).
__device__ __forceinline__ double da_term64(const DADev &d, double q, double d2)
{
    const double dd = __dsqrt_rn(d2);
    if (dd <= d.rs) return __ddiv_rn(q, dd);
    const double t = __ddiv_rn(__dsub_rn(dd, d.rs), d.tw);
    const double sw = __dsub_rn(1.0, __dmul_rn(__dmul_rn(t, t), __dsub_rn(3.0, __dmul_rn(2.0, t))));
    return __ddiv_rn(__dmul_rn(q, sw), dd);
}

// Shell of a counted ion in the taper region (r_s^2 <= d^2 < r_c^2, decided beforehand) from its FP32 squared
// distance d2f; inside the FP32 error of a shell boundary (2^-13 of a shell, far above the 5u of d2f times the
// scale) the reference FP64 formula floor(32 (d^2 - r_s^2) / (r_c^2 - r_s^2)) decides.
__device__ __forceinline__ int da_shell(const DADev &d, float d2f, float4 p, float4 y)
{
    const float kf = (d2f - d.rs2_f) * d.c32_f;
    const float fl = floorf(kf), fr = kf - fl;
    if (fr > 0x1p-13f && fr < 1.0f - 0x1p-13f) return min(31, max(0, (int)fl));
    const double d2 = d2_fp64(p.x, p.y, p.z, y.x, y.y, y.z);
    const int k = (int)floor(__dmul_rn(__ddiv_rn(__dsub_rn(d2, d.rs2), __dsub_rn(d.rc2, d.rs2)), 32.0));
    return min(31, k);
}

// ... is it in the taper region at all (exact)?
__device__ __forceinline__ bool da_in_taper(const DADev &d, float d2f, float4 p, float4 y)
{
    if (d2f > d.rs2_hi) return true;
    if (d2f < d.rs2_lo) return false;
    return d2_fp64(p.x, p.y, p.z, y.x, y.y, y.z) >= d.rs2;
}

__device__ __forceinline__ double silu64(double z)
{
    return __ddiv_rn(z, __dadd_rn(1.0, series_exp(-z)));
}

// ---------------------------------------------------------------------------
// Stage-1 building blocks shared by the sweep kernel and the training-sample kernel.

constexpr int DA_FRS = 33;  // row stride of the per-point shell histograms (32 shells, padded)

// FP32 radial input |p| / R with its error (<= 4u relative: three rounded operations on the squared norm,
// the square root, the division, and fl32(R)).
__device__ __forceinline__ float da_radial32(const DADev &d, float4 p)
{
    return __fdiv_rn(sqrtf(fmaf(p.z, p.z, fmaf(p.y, p.y, p.x * p.x))), d.Rr);
}

__device__ __forceinline__ float silu32(float z)
{
    return __fdiv_rn(z, __fadd_rn(1.0f, expf(-z)));
}

// g(v) in FP32 (BF16 weights held as floats in Wf) with a bound of |g32 - g64|, g64 the reference FP64
// arithmetic on the same weights and exact inputs; v32 carries up to 4u relative error.
// Per layer: FMA chains of n terms err by <= (n+1) u sum |w x|; |silu'| <= 1.1; the FP32 silu adds
// <= 4u |h| + 2u |z| (expf within 2 ulp, one add, one division).
__device__ inline void da_mlp32(const float *Wf, const float *w2n, const float v[DA_NIN], float &g, float &eg)
{
    const float *W1 = Wf, *b1 = Wf + DA_OFF_B1, *W2 = Wf + DA_OFF_W2, *b2 = Wf + DA_OFF_B2, *W3 = Wf + DA_OFF_W3;
    const float ev32 = 4.0f * U32 * fabsf(v[32]);
    float h1[DA_H];
    float mh = 0.f, me = 0.f;
#pragma unroll
    for (int o = 0; o < DA_H; ++o) {
        float z0 = b1[o], z1 = 0.f, M = fabsf(b1[o]);
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            z0 = fmaf(W1[o * DA_NIN + i], v[i], z0);
            z1 = fmaf(W1[o * DA_NIN + i + 1], v[i + 1], z1);
            M = fmaf(fabsf(W1[o * DA_NIN + i]), fabsf(v[i]), M);
            M = fmaf(fabsf(W1[o * DA_NIN + i + 1]), fabsf(v[i + 1]), M);
        }
        z0 = fmaf(W1[o * DA_NIN + 32], v[32], z0);
        M = fmaf(fabsf(W1[o * DA_NIN + 32]), fabsf(v[32]), M);
        const float z = z0 + z1;
        const float ez = 36.0f * U32 * M + fabsf(W1[o * DA_NIN + 32]) * ev32;
        const float h = silu32(z);
        h1[o] = h;
        mh = fmaxf(mh, fabsf(h));
        me = fmaxf(me, 1.1f * ez + 4.0f * U32 * fabsf(h) + 2.0f * U32 * fabsf(z));
    }
    float gs = Wf[DA_OFF_B3], Mg = fabsf(Wf[DA_OFF_B3]), eacc = 0.f;
#pragma unroll 1
    for (int o = 0; o < DA_H; ++o) {
        float z0 = b2[o], z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
        for (int i = 0; i < DA_H; i += 4) {
            z0 = fmaf(W2[o * DA_H + i], h1[i], z0);
            z1 = fmaf(W2[o * DA_H + i + 1], h1[i + 1], z1);
            z2 = fmaf(W2[o * DA_H + i + 2], h1[i + 2], z2);
            z3 = fmaf(W2[o * DA_H + i + 3], h1[i + 3], z3);
        }
        const float z = (z0 + z1) + (z2 + z3);
        const float ez = 68.0f * U32 * (fabsf(b2[o]) + w2n[o] * mh) + w2n[o] * me;
        const float h = silu32(z);
        const float eh = 1.1f * ez + 4.0f * U32 * fabsf(h) + 2.0f * U32 * fabsf(z);
        gs = fmaf(W3[o], h, gs);
        Mg = fmaf(fabsf(W3[o]), fabsf(h), Mg);
        eacc = fmaf(fabsf(W3[o]), eh, eacc);
    }
    g = gs;
    eg = (66.0f * U32 * Mg + eacc) * (1.0f + 0x1p-8f);
}

// Near field of move k (one warp): FP32 sums of q_j / r over counted ions within r_c of the old (0) and the
// trial (1) position, their sums of |q_j| / r, the trial's overlap with a counted ion (exact: the FP64 squared
// distance decides inside the FP32 band), and the largest number of terms one lane added.  Membership in r_c
// is exact the same way.
struct NearOut {
    float ph0, ph1, A0, A1;
    int nt, ovl;
};

constexpr int NF_ST = 125;  // near-field stencil: the 5^3 cells within two of the ion's cell

// Near field of a move (one warp); wsc is this warp's scratch of 2 x 128 ints.  The candidates are the ions
// of the stencil cells whose box lies within the reach of the old position x.  Lane l holds cells
// c = l + 32 u (u < 4) at positions p = 4 l + u; the running count over positions and each position's first
// slot go to wsc, and each candidate finds its cell by a binary search over the running counts.
__device__ inline NearOut da_near_warp(const DADev &d, int g, int B, int Wg, int i, float4 x, float4 a, float lo2, float hi2,
                                       double sig2, int *F0, int *F1, int *wsc)
{
    const int lane = threadIdx.x & 31;
    const int G = d.nf_G;
    const int cx = da_ncell_axis(d, x.x), cy = da_ncell_axis(d, x.y), cz = da_ncell_axis(d, x.z);
    int *pre = wsc, *cst = wsc + 128;  // by position p = 4 lane + u
    __syncwarp();                      // the previous move's readers are done with the scratch
    // lane-local counts of its stencil cells (c = lane + 32 u), then the warp's running sum over all cells
    int cnt4[4], lsum = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        int n = 0, lo = 0;
        if (c < NF_ST) {
            const int ax = cx + c / 25 - 2, ay = cy + (c / 5) % 5 - 2, az = cz + c % 5 - 2;
            if (ax >= 0 && ay >= 0 && az >= 0 && ax < G && ay < G && az < G) {
                const float bx = -d.nf_R + (float)ax * d.nf_edge, by = -d.nf_R + (float)ay * d.nf_edge,
                            bz = -d.nf_R + (float)az * d.nf_edge;
                const float ex = fmaxf(fmaxf(bx - x.x, x.x - (bx + d.nf_edge)), 0.f);
                const float ey = fmaxf(fmaxf(by - x.y, x.y - (by + d.nf_edge)), 0.f);
                const float ez = fmaxf(fmaxf(bz - x.z, x.z - (bz + d.nf_edge)), 0.f);
                if (fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= d.reach2) {
                    const int q = (ax * G + ay) * G + az;
                    lo = __ldg(&d.cell_start[q]);
                    n = __ldg(&d.cell_start[q + 1]) - lo;
                }
            }
        }
        cst[4 * lane + u] = lo;
        cnt4[u] = n;
        lsum += n;
    }
    int incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    {
        int run = incl - lsum;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            run += cnt4[u];
            pre[4 * lane + u] = run;  // candidates in positions 0 .. 4 lane + u
        }
    }
    __syncwarp();
    float ph0 = 0.f, ph1 = 0.f, A0 = 0.f, A1 = 0.f;
    int n0 = 0, n1 = 0, ovl = 0;
    constexpr int U = 4;  // candidates in flight per lane: their loads are issued before any is used
    for (int t0 = 0; t0 < total; t0 += 32 * U) {
        int idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + 32 * u + lane;
            // the first position whose running count exceeds t (pre(-1) = 0 <= t < pre(127) = total)
            int lo_p = -1, hi_p = 127;
#pragma unroll
            for (int step = 0; step < 7; ++step) {
                const int mid = (lo_p + hi_p) >> 1;
                if (pre[mid] <= t) lo_p = mid;
                else hi_p = mid;
            }
            const int before = lo_p < 0 ? 0 : pre[lo_p];
            idx[u] = t < total ? cst[hi_p] + (t - before) : -1;
        }
        int jj[U];
        float4 yy[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            jj[u] = idx[u] >= 0 ? __ldg(&d.cell_ions[idx[u]]) : -1;
            yy[u] = idx[u] >= 0 ? __ldcg(&d.cell_pos[idx[u]]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jj[u];
            if (j < 0 || !da_counted(i, g, B, Wg, j)) continue;
            const float4 y = yy[u];
            const float aq = fabsf(y.w);
            {
                const float dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                bool in = d2 < d.rc2_lo;
                if (!in && !(d2 > d.rc2_hi)) in = d2_fp64(x.x, x.y, x.z, y.x, y.y, y.z) < d.rc2;
                if (in) {
                    const float r = rsqrt_approx(d2);
                    ph0 = fmaf(y.w * da_taper32(d, d2 * r), r, ph0);
                    A0 = fmaf(aq, r, A0);
                    ++n0;
                    if (da_in_taper(d, d2, x, y)) atomicAdd(&F0[da_shell(d, d2, x, y)], (int)y.w);
                }
            }
            {
                const float dx = a.x - y.x, dy = a.y - y.y, dz = a.z - y.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (d2 < lo2) ovl = 1;
                else if (!(d2 > hi2) && d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < sig2) ovl = 1;
                bool in = d2 < d.rc2_lo;
                if (!in && !(d2 > d.rc2_hi)) in = d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < d.rc2;
                if (in) {
                    const float r = rsqrt_approx(d2);
                    ph1 = fmaf(y.w * da_taper32(d, d2 * r), r, ph1);
                    A1 = fmaf(aq, r, A1);
                    ++n1;
                    if (da_in_taper(d, d2, a, y)) atomicAdd(&F1[da_shell(d, d2, a, y)], (int)y.w);
                }
            }
        }
    }
    NearOut o;
    int nt = max(n0, n1);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        ph0 += __shfl_xor_sync(0xffffffffu, ph0, s);
        ph1 += __shfl_xor_sync(0xffffffffu, ph1, s);
        A0 += __shfl_xor_sync(0xffffffffu, A0, s);
        A1 += __shfl_xor_sync(0xffffffffu, A1, s);
        nt = max(nt, __shfl_xor_sync(0xffffffffu, nt, s));
        ovl |= __shfl_xor_sync(0xffffffffu, ovl, s);
    }
    o.ph0 = ph0;
    o.ph1 = ph1;
    o.A0 = A0;
    o.A1 = A1;
    o.nt = nt;
    o.ovl = ovl;
    return o;
}

// Overlap prefilter: does the trial position a of ion i (old position x) overlap a counted ion?  Warp-collective
// over the 5 x 5 x 5 cells around x's cell (edge >= half the reach, so they hold every ion that can lie within
// sigma of a at any time of the sweep); each lane takes up to four cells and their listed ions.  An ion left out
// of a full cell is only a missed rejection: the exact pass finds every overlap.  Returns the same value in every
// lane: 1 when some counted ion certainly overlaps (FP32 squared distance below lo2, or the reference FP64 test
// inside the band).
__device__ inline int da_ovl_warp(const DADev &d, int g, int B, int Wg, int i, float4 x, float4 a, float lo2, float hi2,
                                  double sig2)
{
    const int lane = threadIdx.x & 31;
    const int G = d.nf_G;
    const int cx = da_ncell_axis(d, x.x), cy = da_ncell_axis(d, x.y), cz = da_ncell_axis(d, x.z);
    int ovl = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        if (c >= NF_ST) continue;
        const int ax = cx + c / 25 - 2, ay = cy + (c / 5) % 5 - 2, az = cz + c % 5 - 2;
        if (ax < 0 || ay < 0 || az < 0 || ax >= G || ay >= G || az >= G) continue;
        const float bx = -d.nf_R + (float)ax * d.nf_edge, by = -d.nf_R + (float)ay * d.nf_edge,
                    bz = -d.nf_R + (float)az * d.nf_edge;
        const float ex = fmaxf(fmaxf(bx - a.x, a.x - (bx + d.nf_edge)), 0.f);
        const float ey = fmaxf(fmaxf(by - a.y, a.y - (by + d.nf_edge)), 0.f);
        const float ez = fmaxf(fmaxf(bz - a.z, a.z - (bz + d.nf_edge)), 0.f);
        if (fmaf(ez, ez, fmaf(ey, ey, ex * ex)) > d.ovl_reach2) continue;
        const int q = (ax * G + ay) * G + az;
        const int n = min(__ldg(&d.cell_cnt[q]), d.cap);
        for (int t = 0; t < n && !ovl; ++t) {
            const float4 y = __ldcg(&d.cell_pos[q * d.cap + t]);  // fourth word: the ion's index
            if (!da_counted(i, g, B, Wg, __float_as_int(y.w))) continue;
            const float dx = a.x - y.x, dy = a.y - y.y, dz = a.z - y.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2 < lo2) ovl = 1;
            else if (!(d2 > hi2) && d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z) < sig2) ovl = 1;
        }
    }
    return __any_sync(0xffffffffu, ovl) ? 1 : 0;
}

}  // namespace mcg
