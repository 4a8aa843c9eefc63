// mc_aux.cu -- kernels off the timed sweep path: total energy (initial ledger
// value and drift check), the pair-distance histogram behind g(r), and the
// test hooks for the Philox stream and the FP64 logarithm.
#include <curand_kernel.h>

#include <cstdint>
#include <mutex>

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

}  // namespace mcg

namespace mcg_host {

cudaError_t energy_launch(const float4 *pos, int N, double lB, double *rows, double *out, cudaStream_t st)
{
    mcg::energy_rows<<<(N + mcg::EB - 1) / mcg::EB, mcg::EB, 0, st>>>(pos, N, rows);
    mcg::energy_reduce<<<1, 1024, 0, st>>>(rows, N, lB, out);
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

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

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
        // set-up, once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_rows);
            if (e != cudaSuccess || !ptr) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double *>(ptr);
        }
        rows = g_noalloc_ptr[dev];
    }
    e = mcg_host::energy_launch(static_cast<const float4 *>(pos_q_dev), (int)n, l_B, rows, energy_dev,
                                static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return mcg_host::set_error(MC_ERR_CUDA, cudaGetErrorString(e));
    return MC_OK;
}
