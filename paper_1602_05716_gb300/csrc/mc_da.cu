// mc_da.cu -- delayed acceptance outside the sweep kernel: the per-sweep
// preparation (near-field cell list of the sweep's start positions), the
// surrogate MLP's inference and training kernels (forward,
// backward, weight gradients reduced in a fixed order, Adam with BF16
// rounding of the weights), and the kernel that turns a configuration and
// the chain's own trial moves into training samples (features at the old and
// trial positions, and the far part of the exact energy change).
#include <cstdint>

#include "../../include/mc.h"
#include "mc_da.cuh"

namespace mcg {

// ---------------------------------------------------------------------------
// Per-sweep preparation (stream-ordered before the sweep kernel).

// The sweep's start positions: the buffer of the chain's current sweep count (read on the device, so a
// captured graph stays valid as the count advances).
__device__ __forceinline__ const float4 *start_positions(const ChainDev &ch)
{
    return ch.pos[*ch.sweep & 1];
}

__global__ void da_prep_count(const ChainDev *__restrict__ chp, int N, const DADev *__restrict__ dp, int *cnt,
                              int *cellid)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const DADev &d = *dp;
    const float4 x = start_positions(*chp)[j];
    const int G = d.nf_G;
    const int c = (da_ncell_axis(d, x.x) * G + da_ncell_axis(d, x.y)) * G + da_ncell_axis(d, x.z);
    cellid[j] = c;
    atomicAdd(&cnt[c], 1);
}

// Exclusive scan of the cell counts (one block): cell_start[c] and the scatter cursors.
__global__ void __launch_bounds__(1024) da_prep_scan(const int *__restrict__ cnt, int ncell, int *start, int *fill)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x, per = (ncell + 1023) / 1024;
    const int c0 = min(ncell, tid * per), c1 = min(ncell, c0 + per);
    int s = 0;
    for (int c = c0; c < c1; ++c) s += cnt[c];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - s;
    for (int c = c0; c < c1; ++c) {
        start[c] = run;
        fill[c] = run;
        run += cnt[c];
    }
    if (tid == 1023) start[ncell] = part[1023];
}

__global__ void da_prep_scatter(const ChainDev *__restrict__ chp, int N, const int *__restrict__ cellid, int *fill,
                                int *cell_ions, float4 *cell_pos, int *slot_of)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int slot = atomicAdd(&fill[cellid[j]], 1);
    cell_ions[slot] = j;
    cell_pos[slot] = start_positions(*chp)[j];
    slot_of[j] = slot;
}

// Overlap prefilter: bucket layout of the sweep's start positions (cell q: slots q cap .. q cap + cap - 1, each the
// position with the ion's index in place of its valence, filled in arrival order; the order never matters, the prefilter only asks whether some listed ion overlaps).  cnt must
// be zero on entry; it ends with the number of ions of each cell, possibly above cap (those past it are unlisted).
__global__ void da_prep_bucket(const ChainDev *__restrict__ chp, int N, const DADev *__restrict__ dp, int *cnt,
                               float4 *cell_pos, int *slot_of)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const DADev &d = *dp;
    const float4 x = start_positions(*chp)[j];
    const int G = d.nf_G;
    const int c = (da_ncell_axis(d, x.x) * G + da_ncell_axis(d, x.y)) * G + da_ncell_axis(d, x.z);
    const int t = atomicAdd(&cnt[c], 1);
    if (t < d.cap) {
        const int slot = c * d.cap + t;
        cell_pos[slot] = make_float4(x.x, x.y, x.z, __int_as_float(j));  // the ion's index in the fourth word
        slot_of[j] = slot;
    } else {
        slot_of[j] = -1;
    }
}

// ---------------------------------------------------------------------------
// Surrogate MLP (33-64-64-1, SiLU, BF16 weights, FP32 arithmetic).

constexpr int MT = 256;      // threads per block of the MLP kernels
constexpr int ZS = 2 * DA_H; // stored pre-activations per point (z1 | z2)

__device__ __forceinline__ void load_weights(float *Wf, const unsigned short *w)
{
    for (int q = threadIdx.x; q < DA_NP; q += blockDim.x) Wf[q] = bf16f(__ldg(&w[q]));
    __syncthreads();
}

__device__ __forceinline__ float sigm(float z)
{
    return __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-z)));
}

// Forward pass of one point, keeping z1 and z2.
__device__ float mlp_point(const float *Wf, const float *v, float *z1, float *z2)
{
    float h1[DA_H];
#pragma unroll 4
    for (int o = 0; o < DA_H; ++o) {
        float z = Wf[DA_OFF_B1 + o];
        for (int i = 0; i < DA_NIN; ++i) z = fmaf(Wf[o * DA_NIN + i], v[i], z);
        z1[o] = z;
    }
#pragma unroll
    for (int o = 0; o < DA_H; ++o) h1[o] = z1[o] * sigm(z1[o]);
    float g = Wf[DA_OFF_B3];
#pragma unroll 1
    for (int o = 0; o < DA_H; ++o) {
        float z = Wf[DA_OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < DA_H; ++i) z = fmaf(Wf[DA_OFF_W2 + o * DA_H + i], h1[i], z);
        z2[o] = z;
        g = fmaf(Wf[DA_OFF_W3 + o], z * sigm(z), g);
    }
    return g;
}

// g at n points (V: n x 33); Z (n x 128) optional.
__global__ void __launch_bounds__(MT) mlp_forward_kernel(const unsigned short *__restrict__ w, const float *__restrict__ V,
                                                         long long n, float *__restrict__ G, float *__restrict__ Z)
{
    __shared__ float Wf[DA_NP];
    load_weights(Wf, w);
    const long long p = (long long)blockIdx.x * MT + threadIdx.x;
    if (p >= n) return;
    float v[DA_NIN], z1[DA_H], z2[DA_H];
    for (int i = 0; i < DA_NIN; ++i) v[i] = V[p * DA_NIN + i];
    G[p] = mlp_point(Wf, v, z1, z2);
    if (Z)
        for (int o = 0; o < DA_H; ++o) {
            Z[p * ZS + o] = z1[o];
            Z[p * ZS + DA_H + o] = z2[o];
        }
}

// Backward deltas of the pair loss (1/n_total) sum (g(v1) - g(v0) - y)^2.  Points are interleaved
// (2p = old position, 2p+1 = trial).  D per point: dz1 (64), dz2 (64), dg; loss partials per block.
__global__ void __launch_bounds__(MT) mlp_backward_kernel(const unsigned short *__restrict__ w, const float *__restrict__ Z,
                                                          const float *__restrict__ G, const float *__restrict__ Y,
                                                          long long npairs, float inv_n, float *__restrict__ D,
                                                          double *__restrict__ loss_part)
{
    __shared__ float Wf[DA_NP];
    __shared__ double red[MT];
    load_weights(Wf, w);
    const long long p = (long long)blockIdx.x * MT + threadIdx.x;
    double l2 = 0.0;
    if (p < npairs) {
        const float r = (G[2 * p + 1] - G[2 * p]) - Y[p];
        l2 = (double)r * (double)r;
        for (int side = 0; side < 2; ++side) {
            const long long pt = 2 * p + side;
            const float dg = (side ? 2.0f : -2.0f) * r * inv_n;
            const float *z = Z + pt * ZS;
            float *dd = D + pt * (ZS + 1);
            float dz2[DA_H];
#pragma unroll
            for (int o = 0; o < DA_H; ++o) {
                const float zz = z[DA_H + o], sg = sigm(zz);
                dz2[o] = dg * Wf[DA_OFF_W3 + o] * (sg * (1.0f + zz * (1.0f - sg)));
                dd[DA_H + o] = dz2[o];
            }
#pragma unroll 1
            for (int i = 0; i < DA_H; ++i) {
                float dh = 0.f;
#pragma unroll
                for (int o = 0; o < DA_H; ++o) dh = fmaf(dz2[o], Wf[DA_OFF_W2 + o * DA_H + i], dh);
                const float zz = z[i], sg = sigm(zz);
                dd[i] = dh * (sg * (1.0f + zz * (1.0f - sg)));
            }
            dd[ZS] = dg;
        }
    }
    red[threadIdx.x] = l2;
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// Weight gradients: per block, a fixed range of points; one partial per parameter and block.
constexpr int PC = 32;                            // points staged per step
constexpr int PPT = (DA_NP + MT - 1) / MT;        // parameters per thread (26)
__global__ void __launch_bounds__(MT) mlp_wgrad_kernel(const float *__restrict__ V, const float *__restrict__ Z,
                                                       const float *__restrict__ D, long long npts, long long per_block,
                                                       float *__restrict__ part)
{
    __shared__ float sv[PC][DA_NIN], sh1[PC][DA_H], sh2[PC][DA_H], sd1[PC][DA_H], sd2[PC][DA_H], sdg[PC];
    const int tid = threadIdx.x;
    float acc[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) acc[u] = 0.f;
    const long long p0 = (long long)blockIdx.x * per_block, p1 = min(npts, p0 + per_block);
    for (long long base = p0; base < p1; base += PC) {
        const int np = (int)min((long long)PC, p1 - base);
        __syncthreads();
        for (int e = tid; e < np * DA_NIN; e += MT) sv[e / DA_NIN][e % DA_NIN] = V[(base + e / DA_NIN) * DA_NIN + e % DA_NIN];
        for (int e = tid; e < np * DA_H; e += MT) {
            const int q = e / DA_H, o = e % DA_H;
            const float z1 = Z[(base + q) * ZS + o], z2 = Z[(base + q) * ZS + DA_H + o];
            sh1[q][o] = z1 * sigm(z1);
            sh2[q][o] = z2 * sigm(z2);
            sd1[q][o] = D[(base + q) * (ZS + 1) + o];
            sd2[q][o] = D[(base + q) * (ZS + 1) + DA_H + o];
        }
        for (int e = tid; e < np; e += MT) sdg[e] = D[(base + e) * (ZS + 1) + ZS];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int q = tid + u * MT;
            if (q >= DA_NP) continue;
            float a = acc[u];
            if (q < DA_OFF_B1) {
                const int o = q / DA_NIN, i = q % DA_NIN;
                for (int t = 0; t < np; ++t) a = fmaf(sd1[t][o], sv[t][i], a);
            } else if (q < DA_OFF_W2) {
                const int o = q - DA_OFF_B1;
                for (int t = 0; t < np; ++t) a += sd1[t][o];
            } else if (q < DA_OFF_B2) {
                const int o = (q - DA_OFF_W2) / DA_H, i = (q - DA_OFF_W2) % DA_H;
                for (int t = 0; t < np; ++t) a = fmaf(sd2[t][o], sh1[t][i], a);
            } else if (q < DA_OFF_W3) {
                const int o = q - DA_OFF_B2;
                for (int t = 0; t < np; ++t) a += sd2[t][o];
            } else if (q < DA_OFF_B3) {
                const int o = q - DA_OFF_W3;
                for (int t = 0; t < np; ++t) a = fmaf(sdg[t], sh2[t][o], a);
            } else {
                for (int t = 0; t < np; ++t) a += sdg[t];
            }
            acc[u] = a;
        }
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        const int q = tid + u * MT;
        if (q < DA_NP) part[(long long)blockIdx.x * DA_NP + q] = acc[u];
    }
}

__global__ void mlp_reduce_kernel(const float *__restrict__ part, int nparts, float *__restrict__ grad)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= DA_NP) return;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += part[(long long)b * DA_NP + q];
    grad[q] = s;
}

__device__ __forceinline__ unsigned short f32_to_bf16(float f)
{
    const unsigned u = __float_as_uint(f);
    return (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

// Adam on FP32 master weights; the BF16 copy (round to nearest even) is what the forward pass uses.
__global__ void adam_kernel(float *p, float *m, float *v, const float *__restrict__ g, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, unsigned short *wbf)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= DA_NP) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float pq = p[q] - lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
    p[q] = pq;
    wbf[q] = f32_to_bf16(pq);
}

// ---------------------------------------------------------------------------
// Training samples from a configuration: for the S moves of each group (the chain's own trial moves of its
// next sweep), the features at the old and trial positions, the near-field potentials and the exact pair
// sum, all over the configuration as it stands; y = exact sum - (phi_trial - phi_old), the far part the
// MLP learns.  One block per group at a time.
struct SampleSmem {
    float4 own[S], trial[S], tile[S];
    int Fr[2 * S * DA_FRS];
    float ph0[S], ph1[S], ex[S], mn[S];
    int ovl[S];
    int wsc[T / 32][256];
};

__global__ void __launch_bounds__(T, 1) da_sample_kernel(const ChainDev *__restrict__ chp, const DADev *__restrict__ dp,
                                                         int g0, int g1, float *__restrict__ V, float *__restrict__ Y,
                                                         unsigned char *__restrict__ valid)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SampleSmem &sm = *reinterpret_cast<SampleSmem *>(smraw);
    const ChainDev &ch = *chp;
    const DADev &d = *dp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = ch.N, B = ch.B, Wg = min(d.W, B - 1);
    const unsigned long long s = *ch.sweep;
    const float4 *P = ch.pos[s & 1];
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        const int k0 = g * S, nk = min(S, N - k0);
        __syncthreads();
        if (tid < S) {
            const int k = tid;
            if (k < nk) {
                const float4 x = P[k0 + k];
                const uint4 w = move_draws(ch, s * (unsigned long long)N + (unsigned long long)(k0 + k), 0u);
                sm.own[k] = x;
                sm.trial[k] = make_float4(trial_coord(x.x, w.x, ch.D), trial_coord(x.y, w.y, ch.D),
                                          trial_coord(x.z, w.z, ch.D), x.w);
            } else {
                sm.own[k] = make_float4(-1.0e6f, -1.0e6f, -1.0e6f, 0.f);
                sm.trial[k] = sm.own[k];
            }
            sm.ex[k] = 0.f;
            sm.mn[k] = 3.0e38f;
        }
        for (int q = tid; q < 2 * S * DA_FRS; q += T) sm.Fr[q] = 0;
        __syncthreads();
        // near field and shell histograms (warp per move)
        for (int k = warp; k < nk; k += T / 32) {
            const NearOut o = da_near_warp(d, g, B, Wg, k0 + k, sm.own[k], sm.trial[k], ch.sig2_lo, ch.sig2_hi, ch.sig2,
                                           sm.Fr + k * DA_FRS, sm.Fr + (S + k) * DA_FRS, sm.wsc[warp]);
            if (lane == 0) {
                sm.ph0[k] = o.ph0;
                sm.ph1[k] = o.ph1;
                sm.ovl[k] = o.ovl;
            }
        }
        // exact pair sums over every other ion (thread: move tid & (S-1), half of each tile)
        {
            const int k = tid & (S - 1), h = tid >> 7;
            const float4 a = sm.trial[k], b = sm.own[k];
            const float3 b3 = make_float3(b.x, b.y, b.z), d3 = make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
            float sum = 0.f, Tt = 0.f, Pp = 0.f, mn = 3.0e38f;
            for (int J = 0; J < B; ++J) {
                __syncthreads();
                if (tid < S) sm.tile[tid] = (J * S + tid < N) ? P[J * S + tid] : make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
                __syncthreads();
                for (int l = h; l < S; l += 2) {
                    if (J * S + l == k0 + k) continue;
                    pair_far(b3, d3, sm.tile[l], sum, Tt, Pp, mn);
                }
            }
            atomicAdd(&sm.ex[k], sum);
            atomicMin(reinterpret_cast<int *>(&sm.mn[k]), __float_as_int(mn));
        }
        __syncthreads();
        if (tid < nk) {
            const int k = tid;
            const long long m = (long long)(k0 + k);
            for (int i = 0; i < 32; ++i) {
                V[m * 66 + i] = (float)sm.Fr[k * DA_FRS + i] * 0.25f;
                V[m * 66 + 33 + i] = (float)sm.Fr[(S + k) * DA_FRS + i] * 0.25f;
            }
            V[m * 66 + 32] = da_radial32(d, sm.own[k]);
            V[m * 66 + 33 + 32] = da_radial32(d, sm.trial[k]);
            const float4 a = sm.trial[k];
            const double r2 = (double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z;
            const bool ok = !(r2 > ch.Rc2) && !sm.ovl[k] && sm.mn[k] >= (float)ch.sig2;
            valid[m] = ok ? 1 : 0;
            Y[m] = sm.ex[k] - (sm.ph1[k] - sm.ph0[k]);
        }
    }
}

}  // namespace mcg

namespace mcg_host {

cudaError_t da_prep_launch(const mcg::ChainDev *chd, int N, const mcg::DADev *dd, int ncell, int *cnt, int *cellid,
                           int *start, int *fill, int *cell_ions, float4 *cell_pos, int *slot_of, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncell, st)) != cudaSuccess) return e;
    mcg::da_prep_count<<<(N + 255) / 256, 256, 0, st>>>(chd, N, dd, cnt, cellid);
    mcg::da_prep_scan<<<1, 1024, 0, st>>>(cnt, ncell, start, fill);
    mcg::da_prep_scatter<<<(N + 255) / 256, 256, 0, st>>>(chd, N, cellid, fill, cell_ions, cell_pos, slot_of);
    return cudaGetLastError();
}

cudaError_t da_prep_bucket_launch(const mcg::ChainDev *chd, int N, const mcg::DADev *dd, int ncell, int *cnt,
                                  float4 *cell_pos, int *slot_of, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncell, st)) != cudaSuccess) return e;
    mcg::da_prep_bucket<<<(N + 255) / 256, 256, 0, st>>>(chd, N, dd, cnt, cell_pos, slot_of);
    return cudaGetLastError();
}

cudaError_t da_sample_launch(const mcg::ChainDev *ch, const mcg::DADev *dd, int B, int grid, float *V, float *Y,
                             unsigned char *valid, cudaStream_t st)
{
    const size_t sm = sizeof(mcg::SampleSmem);
    cudaError_t e = cudaFuncSetAttribute(mcg::da_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    mcg::da_sample_kernel<<<grid, mcg::T, sm, st>>>(ch, dd, 0, B, V, Y, valid);
    return cudaGetLastError();
}

cudaError_t mlp_forward_launch(const unsigned short *w, const float *V, long long n, float *G, float *Z, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    mcg::mlp_forward_kernel<<<(unsigned)((n + mcg::MT - 1) / mcg::MT), mcg::MT, 0, st>>>(w, V, n, G, Z);
    return cudaGetLastError();
}

cudaError_t mlp_backward_launch(const unsigned short *w, const float *Z, const float *G, const float *Y, long long npairs,
                                float inv_n, float *D, double *loss_part, cudaStream_t st)
{
    mcg::mlp_backward_kernel<<<(unsigned)((npairs + mcg::MT - 1) / mcg::MT), mcg::MT, 0, st>>>(w, Z, G, Y, npairs, inv_n, D,
                                                                                             loss_part);
    return cudaGetLastError();
}

cudaError_t mlp_wgrad_launch(const float *V, const float *Z, const float *D, long long npts, int nblocks, float *part,
                             float *grad, cudaStream_t st)
{
    const long long per = (npts + nblocks - 1) / nblocks;
    mcg::mlp_wgrad_kernel<<<nblocks, mcg::MT, 0, st>>>(V, Z, D, npts, per, part);
    mcg::mlp_reduce_kernel<<<(mcg::DA_NP + 255) / 256, 256, 0, st>>>(part, nblocks, grad);
    return cudaGetLastError();
}

cudaError_t adam_launch(float *p, float *m, float *v, const float *g, float lr, float b1, float b2, float eps, float bc1,
                        float bc2, unsigned short *wbf, cudaStream_t st)
{
    mcg::adam_kernel<<<(mcg::DA_NP + 255) / 256, 256, 0, st>>>(p, m, v, g, lr, b1, b2, eps, bc1, bc2, wbf);
    return cudaGetLastError();
}

}  // namespace mcg_host
