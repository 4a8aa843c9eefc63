// mc_aux.cu -- kernels off the timed sweep path: total energy (initial ledger
// value and drift check), the pair-distance histogram behind g(r), and the
// test hooks for the Philox stream and the FP64 logarithm.
#include <curand_kernel.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/mc.h"
#include "mc_device.cuh"

namespace mcg {

constexpr int EB = 256;  // rows per energy / histogram block (one per thread)

// Row sums of the Coulomb energy: out[i] = q_i * sum_{j != i} q_j / r_ij with
// FP32 terms (rsqrt.approx) promoted to FP64 per 256-column tile.  Every
// ordered pair is visited, so E = (l_B / 2) sum_i out[i] (Sec. 5.2 monitors the
// total energy of the system).
__global__ void __launch_bounds__(EB) energy_rows(const float4 *__restrict__ pos, int N, double *__restrict__ out)
{
    __shared__ float4 tile[EB];
    const int i = blockIdx.x * EB + threadIdx.x;
    const float4 a = i < N ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    double row = 0.0;
    for (int j0 = 0; j0 < N; j0 += EB) {
        const int j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < N ? pos[j] : make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
        __syncthreads();
        float part = 0.f;
#pragma unroll 8
        for (int l = 0; l < EB; ++l) {
            const float4 y = tile[l];
            const float dx = a.x - y.x, dy = a.y - y.y, dz = a.z - y.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float t = (j0 + l == i) ? 0.f : y.w * rsqrt_approx(d2);
            part += t;
        }
        row += (double)part;
        __syncthreads();
    }
    if (i < N) out[i] = (double)a.w * row;
}

// Deterministic single-block sum: E = (l_B / 2) sum_i rows[i].
__global__ void __launch_bounds__(1024) energy_reduce(const double *__restrict__ rows, int N, double lB,
                                                       double *__restrict__ out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += 1024) s += rows[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * lB * red[0];
}

// Pair-distance histogram (Sec. 5.2, Fig. PCF).  Rows i with
// ((double)x^2 + (double)y^2) + (double)z^2 <= lim2 (all rows when use_lim == 0);
// every j != i; bin = floor(sqrt(d2) / dr) in FP64 from the FP32 centres; an
// FP32 prefilter d2f > rmax2_hi skips pairs that are certainly out of range.
__global__ void __launch_bounds__(EB) gr_hist(const float4 *__restrict__ pos, int N, int n_bins, double dr,
                                              float rmax2_hi, int use_lim, double lim2,
                                              unsigned long long *__restrict__ counts)
{
    extern __shared__ unsigned long long hist[];  // 3 * n_bins
    __shared__ float4 tile[EB];
    for (int b = threadIdx.x; b < 3 * n_bins; b += EB) hist[b] = 0ull;
    const int i = blockIdx.x * EB + threadIdx.x;
    float4 a = make_float4(-1.0e6f, -1.0e6f, -1.0e6f, 0.f);
    bool row_on = false;
    if (i < N) {
        a = pos[i];
        row_on = true;
        if (use_lim) {
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn((double)a.x, (double)a.x), __dmul_rn((double)a.y, (double)a.y)),
                                        __dmul_rn((double)a.z, (double)a.z));
            row_on = !(r2 > lim2);
        }
    }
    __syncthreads();
    for (int j0 = 0; j0 < N; j0 += EB) {
        const int j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < N ? pos[j] : make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
        __syncthreads();
        if (row_on) {
            for (int l = 0; l < EB; ++l) {
                const float4 y = tile[l];
                const float dx = a.x - y.x, dy = a.y - y.y, dz = a.z - y.z;
                const float d2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (d2f > rmax2_hi || j0 + l == i || j0 + l >= N) continue;
                const double r = __dsqrt_rn(d2_fp64(a.x, a.y, a.z, y.x, y.y, y.z));
                const double fb = floor(__ddiv_rn(r, dr));
                if (fb >= (double)n_bins) continue;
                const int cls = (a.w > 0.f && y.w > 0.f) ? 0 : ((a.w < 0.f && y.w < 0.f) ? 2 : 1);
                atomicAdd(&hist[cls * n_bins + (int)fb], 1ull);
            }
        }
        __syncthreads();
    }
    for (int b = threadIdx.x; b < 3 * n_bins; b += EB)
        if (hist[b]) atomicAdd(&counts[b], hist[b]);
}

// ---------------------------------------------------------------------------
// Accurate total energy (initial ledger, mc_energy's recomputation, the periodic drift check):
// E = l_B sum_{i<j} q_i q_j / r_ij with every term in float-float arithmetic.  The coordinate differences are
// exact (TwoSum), the squared distance is a float-float sum of exact squares (FMA TwoProduct), 1/r is one Newton
// step r0 (1 + (1 - d2 r0^2) / 2) from rsqrt.approx with the residual formed from the exact square of r0, so a
// term's relative error is about 1.5 (2^-22.9)^2 + a few 2^-48 (~2e-14) instead of the FP32 form's ~2^-21.
// Sums: float-float over 64 columns, FP64 per row tile, a fixed tree per block, the blocks' partials in order.
// The upper triangle is cut into pairs of row tiles {b, B-1-b} (equal work, B + 1 column tiles) and each pair into
// C column classes; B and C depend on N only, so the result does not depend on the device.
constexpr int ET = 128;             // rows per row tile
constexpr int EFF_TARGET_BLOCKS = 1216;

__host__ __device__ inline int eff_row_pairs(int N)
{
    const int B = (N + ET - 1) / ET;
    return (B + 1) / 2;
}

__host__ __device__ inline int eff_classes(int N)
{
    const int B = (N + ET - 1) / ET, P = (B + 1) / 2;
    int C = (EFF_TARGET_BLOCKS + P - 1) / P;
    return C < 1 ? 1 : (C > B + 1 ? B + 1 : C);
}

__device__ __forceinline__ void ff_sum(float a, float b, float &s, float &e)  // Knuth's TwoSum
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ff_sq(float h, float &p, float &e)  // h^2 = p + e exactly
{
    p = __fmul_rn(h, h);
    e = __fmaf_rn(h, h, -p);
}

// q_j / |a - y| as th + tl.
__device__ __forceinline__ void ff_term(const float4 a, const float4 y, float &th, float &tl)
{
    float hx, lx, hy, ly, hz, lz;
    ff_sum(a.x, -y.x, hx, lx);
    ff_sum(a.y, -y.y, hy, ly);
    ff_sum(a.z, -y.z, hz, lz);
    float px, ex, py, ey, pz, ez;
    ff_sq(hx, px, ex);
    ff_sq(hy, py, ey);
    ff_sq(hz, pz, ez);
    float s1, e1, s2, e2;
    ff_sum(px, py, s1, e1);
    ff_sum(s1, pz, s2, e2);
    float low = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(ex, ey)), ez);
    low = __fmaf_rn(__fmul_rn(2.0f, hx), lx, low);
    low = __fmaf_rn(__fmul_rn(2.0f, hy), ly, low);
    low = __fmaf_rn(__fmul_rn(2.0f, hz), lz, low);
    const float dh = __fadd_rn(s2, low);                  // Fast2Sum: |s2| >= |low|
    const float dl = __fsub_rn(low, __fsub_rn(dh, s2));
    const float r0 = rsqrt_approx(dh);
    float q0, q1;
    ff_sq(r0, q0, q1);
    float t = __fmaf_rn(-dh, q0, 1.0f);
    t = __fmaf_rn(-dh, q1, t);
    t = __fmaf_rn(-dl, q0, t);
    const float rl = __fmul_rn(__fmul_rn(0.5f, r0), t);
    th = __fmul_rn(y.w, r0);
    tl = __fmaf_rn(y.w, rl, __fmaf_rn(y.w, r0, -th));
}

// Positions: pos0, or, when sweep is non-null, the buffer of the chain's current state pos[*sweep & 1] (read on the
// device, so a captured graph replays correctly whatever the sweep count).
__global__ void __launch_bounds__(2 * ET) energy_ff_part(const float4 *pos0, const float4 *pos1,
                                                          const unsigned long long *sweep, int N,
                                                          double *__restrict__ part)
{
    __shared__ float4 tile[ET];
    const float4 *__restrict__ pos = (sweep && (*sweep & 1ull)) ? pos1 : pos0;
    __shared__ double red[2 * ET];
    const int B = (N + ET - 1) / ET, P = (B + 1) / 2, C = eff_classes(N);
    const int b = blockIdx.x / C, c = blockIdx.x % C;
    const int r = threadIdx.x & (ET - 1), h = threadIdx.x >> 7;
    double tot = 0.0;
    for (int side = 0; side < 2; ++side) {
        const int I = side == 0 ? b : B - 1 - b;
        if (side == 1 && I == b) break;  // the middle row tile of an odd B
        const int i = I * ET + r;
        const float4 a = i < N ? __ldg(&pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        double row = 0.0;
        for (int J = I + c; J < B; J += C) {
            __syncthreads();
            if (threadIdx.x < ET) {
                const int j = J * ET + threadIdx.x;
                tile[threadIdx.x] = j < N ? __ldg(&pos[j]) : make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
            }
            __syncthreads();
            if (i >= N) continue;
            float ah = 0.f, al = 0.f;
            const int l0 = h * (ET / 2);
            if (J == I) {
                for (int l = l0; l < l0 + ET / 2; ++l) {
                    if (l <= r) continue;  // strictly upper: j > i
                    float th, tl, s, e;
                    ff_term(a, tile[l], th, tl);
                    ff_sum(ah, th, s, e);
                    ah = s;
                    al = __fadd_rn(al, __fadd_rn(e, tl));
                }
            } else {
#pragma unroll 4
                for (int l = l0; l < l0 + ET / 2; ++l) {
                    float th, tl, s, e;
                    ff_term(a, tile[l], th, tl);
                    ff_sum(ah, th, s, e);
                    ah = s;
                    al = __fadd_rn(al, __fadd_rn(e, tl));
                }
            }
            row = __dadd_rn(row, __dadd_rn((double)ah, (double)al));
        }
        tot = __dadd_rn(tot, __dmul_rn((double)a.w, row));
    }
    red[threadIdx.x] = tot;
    __syncthreads();
    for (int w = ET; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
    (void)P;
}

// E = l_B sum of the partials in order; optionally the drift |ledger - E| folded into (last, max, count).
__global__ void energy_ff_reduce(const double *__restrict__ part, int n_part, double lB, double *__restrict__ out,
                                 const double *__restrict__ ledger, double *__restrict__ drift)
{
    __shared__ double red[256];
    double s = 0.0;
    const int per = (n_part + 255) / 256;
    for (int k = threadIdx.x * per; k < min(n_part, (int)(threadIdx.x + 1) * per); ++k) s = __dadd_rn(s, part[k]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double E = __dmul_rn(lB, red[0]);
        *out = E;
        if (drift) {
            const double d = fabs(__dsub_rn(*ledger, E));
            drift[0] = d;
            drift[1] = fmax(drift[1], d);
            drift[2] = __dadd_rn(drift[2], 1.0);
        }
    }
}

// ---------------------------------------------------------------------------
// Unit-rate probes behind the ALU roofline (mc_unit_rates): every thread runs UR_CHAINS independent chains of one
// operation, 64 warps per SM (8 blocks of 256 threads at <= 32 registers), and block 0's thread 0 reads clock64
// around the loop.  Rates are operations per SM clock.
constexpr int UR_CHAINS = 8;

__global__ void __launch_bounds__(256, 8) rate_rsqrt(int iters, float *out, long long *cyc)
{
    float x[UR_CHAINS];
#pragma unroll
    for (int q = 0; q < UR_CHAINS; ++q) x[q] = 1.5f + 1e-6f * (float)(threadIdx.x + q);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < UR_CHAINS; ++q) {
            float r;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[q]));
            x[q] = r + 0.5f;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < UR_CHAINS; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(256, 8) rate_ffma2(int iters, float *out, long long *cyc)
{
    f32x2 a[UR_CHAINS];
#pragma unroll
    for (int q = 0; q < UR_CHAINS; ++q) a[q] = pk2(1.f + 1e-7f * (float)(threadIdx.x * q), 1.f - 1e-7f * (float)q);
    const f32x2 b = pk2(0.9999f, 0.9998f), c = pk2(1e-6f, 2e-6f);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < UR_CHAINS; ++q) {
            f32x2 r;
            asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a[q]), "l"(b), "l"(c));
            a[q] = r;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < UR_CHAINS; ++q) {
        float u, v;
        upk2(a[q], u, v);
        s += u + v;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void philox_test(const uint4 *__restrict__ ctr, const uint2 *__restrict__ key, int n, uint4 *out_lib,
                            uint4 *out_curand)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out_lib[t] = philox4x32_10(ctr[t], key[t]);
    out_curand[t] = curand_Philox4x32_10(ctr[t], key[t]);
}

__global__ void log_test(const double *__restrict__ u, int n, double *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = series_log(u[t]);
}

// ---------------------------------------------------------------------------
// Positions from the host (mc_set_positions) checked and packed on the device.  The checks are the library's
// validation rule in FP64, operation for operation (no contraction): |r|^2 = (x^2 + y^2) + z^2 <= Rc^2 for the wall,
// d^2 = (dx^2 + dy^2) + dz^2 >= sigma^2 for every pair.  Pairs are found through a bucket grid of m^3 cells of edge
// >= sigma (the 27 cells around an ion's cell hold every ion closer than sigma); a cell holds at most cap ions,
// cap = k^3 for sub-cubes of diagonal below sigma, so a full cell proves an overlap by itself.  err is a 64-bit
// key: all ones for none, (1 << 62) | i for ion i outside the wall, (2 << 62) | (i << 31) | j for the pair (j < i), the
// smallest key found; (3 << 62) for a full cell.

__device__ __forceinline__ long long vcell(double v, double Rc, double edge, long long m)
{
    long long c = (long long)floor(__ddiv_rn(__dadd_rn(v, Rc), edge));
    return c < 0 ? 0 : (c >= m ? m - 1 : c);
}

__global__ void pos_bin(const float *__restrict__ xyz, int N, double Rc, double edge, int m, int cap, int *cnt,
                        int *ids, unsigned long long *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    if (!(r2 <= __dmul_rn(Rc, Rc))) atomicMin(err, (1ull << 62) | (unsigned long long)i);
    const long long c = (vcell(x, Rc, edge, m) * m + vcell(y, Rc, edge, m)) * m + vcell(z, Rc, edge, m);
    const int t = atomicAdd(&cnt[c], 1);
    if (t < cap) ids[c * cap + t] = i;
    else atomicMin(err, 3ull << 62);
}

__global__ void pos_pairs(const float *__restrict__ xyz, int N, double Rc, double edge, int m, int cap, double s2,
                          const int *__restrict__ cnt, const int *__restrict__ ids, unsigned long long *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const long long cx = vcell(x, Rc, edge, m), cy = vcell(y, Rc, edge, m), cz = vcell(z, Rc, edge, m);
    for (long long ax = cx - 1; ax <= cx + 1; ++ax)
        for (long long ay = cy - 1; ay <= cy + 1; ++ay)
            for (long long az = cz - 1; az <= cz + 1; ++az) {
                if (ax < 0 || ay < 0 || az < 0 || ax >= m || ay >= m || az >= m) continue;
                const long long c = (ax * m + ay) * m + az;
                const int n = min(cnt[c], cap);
                for (int t = 0; t < n; ++t) {
                    const int j = ids[c * cap + t];
                    if (j >= i) continue;  // each pair once, from its larger index
                    const double dx = __dsub_rn((double)xyz[3 * i], (double)xyz[3 * j]);
                    const double dy = __dsub_rn((double)xyz[3 * i + 1], (double)xyz[3 * j + 1]);
                    const double dz = __dsub_rn((double)xyz[3 * i + 2], (double)xyz[3 * j + 2]);
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    if (d2 < s2) atomicMin(err, (2ull << 62) | ((unsigned long long)i << 31) | (unsigned long long)j);
                }
            }
}

// Packed positions: (x, y, z) from xyz and the valence kept in the fourth word of dst.
__global__ void pos_pack(const float *__restrict__ xyz, int N, float4 *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], dst[i].w);
}

__global__ void pos_unpack(const float4 *__restrict__ src, int N, float *xyz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 v = src[i];
    xyz[3 * i] = v.x;
    xyz[3 * i + 1] = v.y;
    xyz[3 * i + 2] = v.z;
}

}  // namespace mcg

namespace mcg_host {

// The device-side check of N host positions already copied to xyz (see pos_bin); err receives the key.
cudaError_t pos_check_launch(const float *xyz, int N, double Rc, double edge, int m, int cap, double s2, int *cnt,
                             int *ids, unsigned long long *err, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)m * m * m, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess || N <= 0) return e;
    const int nb = (N + 255) / 256;
    mcg::pos_bin<<<nb, 256, 0, st>>>(xyz, N, Rc, edge, m, cap, cnt, ids, err);
    mcg::pos_pairs<<<nb, 256, 0, st>>>(xyz, N, Rc, edge, m, cap, s2, cnt, ids, err);
    return cudaGetLastError();
}

cudaError_t pos_pack_launch(const float *xyz, int N, float4 *dst, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    mcg::pos_pack<<<(N + 255) / 256, 256, 0, st>>>(xyz, N, dst);
    return cudaGetLastError();
}

cudaError_t pos_unpack_launch(const float4 *src, int N, float *xyz, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    mcg::pos_unpack<<<(N + 255) / 256, 256, 0, st>>>(src, N, xyz);
    return cudaGetLastError();
}

cudaError_t energy_launch(const float4 *pos, int N, double lB, double *rows, double *out, cudaStream_t st)
{
    mcg::energy_rows<<<(N + mcg::EB - 1) / mcg::EB, mcg::EB, 0, st>>>(pos, N, rows);
    mcg::energy_reduce<<<1, 1024, 0, st>>>(rows, N, lB, out);
    return cudaGetLastError();
}

// Number of FP64 partials of the accurate energy of N ions (the caller's scratch).
int energy_ff_parts(int N)
{
    return mcg::eff_row_pairs(N) * mcg::eff_classes(N);
}

// out = accurate total energy of pos0 (sweep == NULL) or of pos[*sweep & 1]; with ledger/drift non-null also the
// drift fold (see energy_ff_reduce).
cudaError_t energy_ff_launch(const float4 *pos0, const float4 *pos1, const unsigned long long *sweep, int N, double lB,
                             double *part, double *out, const double *ledger, double *drift, cudaStream_t st)
{
    const int n = energy_ff_parts(N);
    mcg::energy_ff_part<<<n, 2 * mcg::ET, 0, st>>>(pos0, pos1, sweep, N, part);
    mcg::energy_ff_reduce<<<1, 256, 0, st>>>(part, n, lB, out, ledger, drift);
    return cudaGetLastError();
}

cudaError_t gr_launch(const float4 *pos, int N, int n_bins, double dr, float rmax2_hi, int use_lim, double lim2,
                      unsigned long long *counts, cudaStream_t st)
{
    const size_t sm = sizeof(unsigned long long) * 3 * (size_t)n_bins;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mcg::gr_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    mcg::gr_hist<<<(N + mcg::EB - 1) / mcg::EB, mcg::EB, sm, st>>>(pos, N, n_bins, dr, rmax2_hi, use_lim, lim2, counts);
    return cudaGetLastError();
}

// Unit rates per SM clock at 8, 16, 32 and 64 resident warps per SM (rows), for rsqrt.approx.ftz and packed
// FFMA2 (columns; FFMA2 counted as two FP32 operations).  Host buffers out[8]; blocks synchronously.
cudaError_t unit_rates(int sms, double *out)
{
    float *buf = nullptr;
    long long *cyc = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * (size_t)sms * 8 * 256);
    if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long) * (size_t)sms * 8);
    std::vector<long long> hc((size_t)sms * 8);
    const int iters = 4096;
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind)
        for (int w = 0; w < 4 && e == cudaSuccess; ++w) {
            const int bps = 1 << w, nb = sms * bps;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                if (kind == 0) mcg::rate_rsqrt<<<nb, 256>>>(iters, buf, cyc);
                else mcg::rate_ffma2<<<nb, 256>>>(iters, buf, cyc);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaDeviceSynchronize();
            }
            if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * nb, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) break;
            double mc = 0.0;
            for (int b = 0; b < nb; ++b) mc += (double)hc[b];
            mc /= nb;
            const double ops = 256.0 * bps * iters * mcg::UR_CHAINS * (kind == 0 ? 1.0 : 2.0);
            out[2 * w + kind] = ops / mc;
        }
    cudaFree(buf);
    cudaFree(cyc);
    return e;
}

cudaError_t philox_test_launch(const uint4 *ctr, const uint2 *key, int n, uint4 *out_lib, uint4 *out_curand,
                               cudaStream_t st)
{
    mcg::philox_test<<<(n + 255) / 256, 256, 0, st>>>(ctr, key, n, out_lib, out_curand);
    return cudaGetLastError();
}

cudaError_t log_test_launch(const double *u, int n, double *out, cudaStream_t st)
{
    mcg::log_test<<<(n + 255) / 256, 256, 0, st>>>(u, n, out);
    return cudaGetLastError();
}

}  // namespace mcg_host

// ---------------------------------------------------------------------------
// Allocation-free total energy (mc_total_energy_noalloc).  Some callers cannot
// allocate device memory while they run: code inside a CUDA stream capture
// (allocation calls are not capturable), real-time loops that must not block
// in the allocator, and hosts whose device memory is owned by a pool they may
// not bypass.  For them the row sums of the energy kernels live in one
// file-scope device array instead of a per-handle buffer.  It is loaded with
// the module, so every GPU that loads this library holds it until the process
// exits.
namespace mcg_host {
int set_error(int code, const char *msg);
}

namespace {

constexpr long long NOALLOC_MAX_IONS = 1ll << 20;  // 8 MiB of FP64 row sums
static __device__ __align__(256) double g_noalloc_rows[NOALLOC_MAX_IONS];

// The array's device address belongs to the context the module was loaded into.  A context that is destroyed and
// created anew (cudaDeviceReset, or the primary context released and retained again) may load the module at
// another address, so the cached address is keyed by the context's unique id and looked up again when it changes.
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];
unsigned long long g_noalloc_ctx[NOALLOC_MAX_DEVICES];  // id of the context the address belongs to (0: none)

typedef int (*ctx_get_current_fn)(void **);
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);

// Unique id of the calling thread's current context, 0 when none is current (or the driver lacks the call).
unsigned long long current_ctx_id()
{
    static ctx_get_current_fn get_cur = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<ctx_get_current_fn>(f1);
            get_id = reinterpret_cast<ctx_get_id_fn>(f2);
        }
        looked_up = true;
    }
    if (!get_cur || !get_id) return 0ull;
    void *ctx = nullptr;
    if (get_cur(&ctx) != 0 || !ctx) return 0ull;
    unsigned long long id = 0ull;
    if (get_id(ctx, &id) != 0) return 0ull;
    return id;
}

}  // namespace

extern "C" int mc_total_energy_noalloc(const void *pos_q_dev, int64_t n, double l_B, double *energy_dev, void *stream)
{
    if (!pos_q_dev || !energy_dev) return mcg_host::set_error(MC_ERR_INVALID, "NULL device pointer");
    if (n < 1 || n > NOALLOC_MAX_IONS)
        return mcg_host::set_error(MC_ERR_INVALID, "n out of range: the allocation-free energy handles 1..1048576 ions");
    if (!(l_B >= 0.0) || l_B > 1.0e300) return mcg_host::set_error(MC_ERR_INVALID, "invalid l_B");
    if ((reinterpret_cast<uintptr_t>(pos_q_dev) & 15u) || (reinterpret_cast<uintptr_t>(energy_dev) & 7u))
        return mcg_host::set_error(MC_ERR_INVALID, "misaligned device pointer (positions need 16 bytes, energy 8)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return mcg_host::set_error(MC_ERR_INVALID, "device ordinal too large");
    double *rows = nullptr;
    {
        // set-up, once per device and context, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        const unsigned long long ctx = current_ctx_id();
        if (!g_noalloc_ptr[dev] || ctx == 0ull || ctx != g_noalloc_ctx[dev]) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
            if (e != cudaSuccess) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
            if (cs != cudaStreamCaptureStatusNone)
                return mcg_host::set_error(MC_ERR_INVALID,
                                           "first call on this device (or after a context reset) inside a stream "
                                           "capture: make one call before capturing");
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_rows);
            if (e != cudaSuccess || !ptr) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double *>(ptr);
            g_noalloc_ctx[dev] = current_ctx_id();  // the look-up made the primary context current if none was
        }
        rows = g_noalloc_ptr[dev];
    }
    e = mcg_host::energy_launch(static_cast<const float4 *>(pos_q_dev), (int)n, l_B, rows, energy_dev,
                                static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
    return MC_OK;
}
