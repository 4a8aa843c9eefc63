// Parallel-reduction Metropolis steps: the comparison GPU code of Sec. 4, built as a foil for the sweep kernel.
//
// One launch per trial move, as in Sec. 4's reduction code: the N - 1 pair terms of ion i are
// spread over blocks of 1,024 threads, one pair per thread (Sec. 4's block size); each block reduces its terms and
// leaves its subtotal in global memory, counts itself done with an atomic, and the last block to finish decides
// the move and updates the ion (Sec. 4's global counter of completed blocks; here the last block is the one whose
// increment completes the count, so no thread spins).  A sweep is N such launches in index order (Sec. 2's
// sequential updating), or N launches each moving an ion drawn at random (Sec. 2's random updating), replayed
// from one CUDA graph.
//
// Decisions are those of the exact chain: every term is the FP64 canonical term (IEEE sqrt and division) of the
// sequential definition; the tree sums differ from the canonical sequential sum by less than a proven bound, and a
// move whose tree value lies inside that bound around its threshold is re-summed by the last block in the
// canonical order (1,024-term chunks summed sequentially, chunk sums in order).  Block subtotals go to fixed
// slots instead of an atomic FP64 add, so the run is reproducible.
#include "mc_device.cuh"

namespace mcg {

constexpr int RT = 1024;  // threads per block: one pair term each

struct RedPart {
    double s;  // tree sum of the block's terms
    double a;  // tree sum of their magnitudes
    int ovl;   // any overlap with the trial position
    int pad;
};

__device__ __forceinline__ void block_reduce(double &s, double &a, int &o, double *ws, double *wa, int *wo)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, d));
        a = __dadd_rn(a, __shfl_xor_sync(0xffffffffu, a, d));
        o |= __shfl_xor_sync(0xffffffffu, o, d);
    }
    if (lane == 0) {
        ws[warp] = s;
        wa[warp] = a;
        wo[warp] = o;
    }
    __syncthreads();
    if (warp == 0) {
        s = ws[lane];
        a = wa[lane];
        o = wo[lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, d));
            a = __dadd_rn(a, __shfl_xor_sync(0xffffffffu, a, d));
            o |= __shfl_xor_sync(0xffffffffu, o, d);
        }
    }
}

// The ion that step m of the random updating scheme moves (Sec. 2, selection at random): u = w1 2^32 + w0 from
// the draws of purpose 3 at move index m, ion floor(u N / 2^64).
__device__ __forceinline__ int random_index(const ChainDev &ch, unsigned long long m)
{
    const uint4 w = move_draws(ch, m, 3u);
    const unsigned long long u = ((unsigned long long)w.y << 32) | (unsigned long long)w.x;
    return (int)__umul64hi(u, (unsigned long long)ch.N);
}

// Step t of the cycle held in *sweep: move index m = sweep N + t, the ion t (sequential updating) or the one
// random_index selects (random updating).  Grid: ceil(N / RT) blocks of RT threads.
// cnt: accepted, Metropolis-rejected, overlap-rejected, wall-rejected, re-summed in the canonical order.
__global__ void __launch_bounds__(RT) reduction_move(const ChainDev *__restrict__ chp, float4 *pos, int t,
                                                      int random_scheme, const unsigned long long *sweep,
                                                      RedPart *part, unsigned *count, double *ledger,
                                                      unsigned long long *cnt)
{
    __shared__ double ws[32], wa[32], terms[RT];
    __shared__ int wo[32];
    __shared__ int last;
    const ChainDev &ch = *chp;
    const int tid = threadIdx.x;
    const int N = ch.N;
    const unsigned long long m = *sweep * (unsigned long long)N + (unsigned long long)t;
    const int i = random_scheme ? random_index(ch, m) : t;
    const float4 b = pos[i];
    const uint4 w = move_draws(ch, m, 0u);
    const float4 a = make_float4(trial_coord(b.x, w.x, ch.D), trial_coord(b.y, w.y, ch.D),
                                 trial_coord(b.z, w.z, ch.D), b.w);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn((double)a.x, (double)a.x), __dmul_rn((double)a.y, (double)a.y)),
                                __dmul_rn((double)a.z, (double)a.z));
    const bool wall = r2 > ch.Rc2;  // rejected before any pair (the wall test comes first)
    double s = 0.0, at = 0.0;
    int o = 0;
    const int j = blockIdx.x * RT + tid;
    if (!wall && j < N && j != i) {
        bool ov;
        s = term_fp64(a, b, pos[j], ov, ch.sig2);
        at = fabs(s);
        o = ov ? 1 : 0;
    }
    block_reduce(s, at, o, ws, wa, wo);
    if (tid == 0) {
        part[blockIdx.x] = RedPart{s, at, o, 0};
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: subtotals in block order, then the decision
    __shared__ double dE_sh, thr_sh;
    __shared__ int res_sh;  // 0 accept, 1 Metropolis reject, 2 overlap, 3 wall, -1 re-sum in the canonical order
    if (tid == 0) {
        double S = 0.0, A = 0.0;
        int ov = 0;
        for (int q = 0; q < (int)gridDim.x; ++q) {
            S = __dadd_rn(S, __ldcg(&part[q].s));  // L2: written by other blocks of this launch
            A = __dadd_rn(A, __ldcg(&part[q].a));
            ov |= __ldcg(&part[q].ovl);
        }
        const unsigned ua = w.w >> 8;
        const double thr = (ua == 0u) ? 0.0 : -series_log((double)ua * 0x1p-24);
        const double lq = __dmul_rn(ch.lB, (double)a.w);
        const double dE = __dmul_rn(lq, S);
        int res;
        if (wall) res = OUT_WALL;
        else if (ov) res = OUT_OVERLAP;
        else if (ua == 0u) res = OUT_ACCEPT;
        else {
            // |tree sum - canonical sum| <= (gamma_depth + gamma_N) sum|t| with depth <= 10 + blocks; both products
            // round once more
            const double bnd = fabs(lq) * (double)(N + (int)gridDim.x + 16) * 0x1p-52 * A * (1.0 + 0x1p-30) +
                               0x1p-50 * (fabs(dE) + thr) + 1e-300;
            res = (dE < thr - bnd) ? OUT_ACCEPT : ((dE > thr + bnd) ? OUT_METROPOLIS : -1);
        }
        dE_sh = dE;
        thr_sh = thr;
        res_sh = res;
    }
    __syncthreads();
    if (res_sh < 0) {  // uniform: the canonical FP64 sum of the exact chain
        double total = 0.0;
        for (int c0 = 0; c0 < N; c0 += RT) {
            const int jj = c0 + tid;
            double v = 0.0;
            if (jj < N && jj != i) {
                bool ov;
                v = term_fp64(a, b, pos[jj], ov, ch.sig2);
            }
            terms[tid] = v;
            __syncthreads();
            if (tid == 0) {
                double sc = 0.0;
                const int len = min(RT, N - c0);
                for (int q = 0; q < len; ++q)
                    if (c0 + q != i) sc = __dadd_rn(sc, terms[q]);
                total = __dadd_rn(total, sc);
            }
            __syncthreads();
        }
        if (tid == 0) {
            const double dE = __dmul_rn(__dmul_rn(ch.lB, (double)a.w), total);
            dE_sh = dE;
            res_sh = (dE < thr_sh) ? OUT_ACCEPT : OUT_METROPOLIS;
            atomicAdd(&cnt[4], 1ull);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int res = res_sh;
        if (res == OUT_ACCEPT) {
            pos[i] = a;
            *ledger = __dadd_rn(*ledger, dE_sh);
        }
        cnt[res] += 1ull;
        *count = 0u;  // the next launch (stream order) starts from zero
    }
}

__global__ void reduction_advance(unsigned long long *sweep)
{
    *sweep += 1ull;
}

}  // namespace mcg

namespace mcg_host {

// One cycle: N single-move launches (steps 0..N-1), then the cycle counter.  `part` holds reduction_part_bytes(N).
cudaError_t reduction_sweep_launch(const mcg::ChainDev *chd, float4 *pos, int N, int random_scheme,
                                   unsigned long long *sweep, void *part, unsigned *count, double *ledger,
                                   unsigned long long *cnt, cudaStream_t st)
{
    const int nb = (N + mcg::RT - 1) / mcg::RT;
    mcg::RedPart *pp = static_cast<mcg::RedPart *>(part);
    for (int t = 0; t < N; ++t) {
        mcg::reduction_move<<<nb, mcg::RT, 0, st>>>(chd, pos, t, random_scheme, sweep, pp, count, ledger, cnt);
    }
    mcg::reduction_advance<<<1, 1, 0, st>>>(sweep);
    return cudaGetLastError();
}

size_t reduction_part_bytes(int N)
{
    return sizeof(mcg::RedPart) * (size_t)((N + mcg::RT - 1) / mcg::RT);
}

}  // namespace mcg_host
