// mc_api.cu -- host runtime behind the C ABI of include/mc.h: chain state in
// device memory, input validation, the work schedule of a launch, CUDA-graph
// capture of sweep launches, and the error protocol of the bounded waits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mc.h"
#include "mc_device.cuh"
#include "mc_da.cuh"

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MC_HAVE_NVTX 1
#endif
#endif

namespace mcg_host {
size_t sweep_smem_bytes();
cudaError_t sweep_configure();
cudaError_t sweep_occupancy(int *blocks_per_sm);
cudaError_t sweep_launch(int grid, const mcg::ChainDev *chains, const mcg::Ticket *sched, int n_tickets, mcg::Ctl *ctl,
                         int n_chains, long long n_sweeps, cudaStream_t st, bool pairs, bool help, bool da);
cudaError_t sweep_occupancy_h(int *blocks_per_sm);
cudaError_t sweep_max_clusters(int *n);
int energy_ff_parts(int N);
cudaError_t energy_ff_launch(const float4 *pos0, const float4 *pos1, const unsigned long long *sweep, int N, double lB,
                             double *part, double *out, const double *ledger, double *drift, cudaStream_t st);
cudaError_t gr_launch(const float4 *pos, int N, int n_bins, double dr, float rmax2_hi, int use_lim, double lim2,
                      unsigned long long *counts, cudaStream_t st);
cudaError_t philox_test_launch(const uint4 *ctr, const uint2 *key, int n, uint4 *out_lib, uint4 *out_curand,
                               cudaStream_t st);
cudaError_t log_test_launch(const double *u, int n, double *out, cudaStream_t st);
cudaError_t unit_rates(int sms, double *out);
cudaError_t pos_check_launch(const float *xyz, int N, double Rc, double edge, int m, int cap, double s2, int *cnt,
                             int *ids, unsigned long long *err, cudaStream_t st);
cudaError_t pos_pack_launch(const float *xyz, int N, float4 *dst, cudaStream_t st);
cudaError_t pos_unpack_launch(const float4 *src, int N, float *xyz, cudaStream_t st);
cudaError_t da_prep_launch(const mcg::ChainDev *chd, int N, const mcg::DADev *dd, int ncell, int *cnt, int *cellid,
                           int *start, int *fill, int *cell_ions, float4 *cell_pos, int *slot_of, cudaStream_t st);
cudaError_t da_prep_bucket_launch(const mcg::ChainDev *chd, int N, const mcg::DADev *dd, int ncell, int *cnt,
                                  float4 *cell_pos, int *slot_of, cudaStream_t st);
cudaError_t da_sample_launch(const mcg::ChainDev *ch, const mcg::DADev *dd, int B, int grid, float *V, float *Y,
                             unsigned char *valid, cudaStream_t st);
cudaError_t mlp_forward_launch(const unsigned short *w, const float *V, long long n, float *G, float *Z, cudaStream_t st);
cudaError_t mlp_backward_launch(const unsigned short *w, const float *Z, const float *G, const float *Y, long long npairs,
                                float inv_n, float *D, double *loss_part, cudaStream_t st);
cudaError_t mlp_wgrad_launch(const float *V, const float *Z, const float *D, long long npts, int nblocks, float *part,
                             float *grad, cudaStream_t st);
cudaError_t adam_launch(float *p, float *m, float *v, const float *g, float lr, float b1, float b2, float eps, float bc1,
                        float bc2, unsigned short *wbf, cudaStream_t st);
cudaError_t reduction_sweep_launch(const mcg::ChainDev *chd, float4 *pos, int N, int random_scheme,
                                   unsigned long long *sweep, void *part, unsigned *count, double *ledger,
                                   unsigned long long *cnt, cudaStream_t st);
size_t reduction_part_bytes(int N);
}  // namespace mcg_host

namespace {

thread_local std::string g_err;

// One NVTX range per entry point: named spans on the host timeline of Nsight tools when one is attached, a few
// nanoseconds otherwise (NVTX v3 loads no tool library unless a tool asks for it).
struct Range {
    explicit Range(const char *name)
    {
#ifdef MC_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range()
    {
#ifdef MC_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    } while (0)

struct Chain {
    int N = 0, B = 0;
    double sigma = 1, lB = 0, R = 1, h = 0;
    uint64_t seed = 0;
    uint32_t chain_id = 0;
    std::vector<float> q;        // host copy of the valences
    float4 *pos[2] = {nullptr, nullptr};  // positions after sweep v live in pos[(v + 1) & 1]
    unsigned long long *flags = nullptr;
    unsigned long long *bits = nullptr;
    unsigned char *slab = nullptr;  // ledger, ledger_seq, stats, sweep, energy out
    double *ledger = nullptr;
    unsigned long long *ledger_seq = nullptr;
    unsigned long long *stats = nullptr;
    unsigned long long *sweep = nullptr;
    double *e_out = nullptr;
    double *eparts = nullptr;    // partial sums of the accurate energy (energy_ff_parts(N) doubles)
    double *drift = nullptr;     // periodic drift check: last |ledger - E|, its maximum, number of checks
    mcg::MoveRec *rec = nullptr;
    long long rec_cap = 0;
    mcg::TraceRec *trace = nullptr;
    long long trace_cap = 0;
    unsigned long long rec_sweep0 = 0;
    double *eser = nullptr;      // energy series (mc_energy_series_enable)
    long long eser_cap = 0;
    unsigned long long eser_sweep0 = 0;
    uint64_t sweeps = 0;         // host mirror of *sweep
    uint64_t sweep_base = 0;     // sweep count when the positions were last set from the host
    float4 *cur() const { return pos[sweeps & 1]; }
    // delayed acceptance (mc_set_surrogate)
    bool da = false;
    bool pf = false;              // the DA state is an overlap prefilter (mc_set_overlap_prefilter)
    int da_k = 1;                 // sweeps per launch its cell list was sized for
    mcg::DADev hda{};             // host copy of the device descriptor
    mcg::DADev *dda = nullptr;    // device descriptor
    unsigned short *d_w = nullptr;
    float *d_w2n = nullptr;
    int *d_cell_start = nullptr, *d_cell_ions = nullptr, *d_slot_of = nullptr, *d_cnt = nullptr, *d_cellid = nullptr;
    int *d_fill = nullptr;
    float4 *d_cell_pos = nullptr;
    // mc_set_positions / mc_get_positions on the device: xyz staging (3N floats), the check's bucket grid, its key
    float *d_xyz = nullptr;
    int *d_vcnt = nullptr, *d_vids = nullptr;
    unsigned long long *d_verr = nullptr;
    int vm = 0, vcap = 0;
    int ncell = 0;
};

struct GraphKey {
    long long n;
    int grid;
    int policy;
    int pairs;
    long long drift;
    bool operator<(const GraphKey &o) const
    {
        if (n != o.n) return n < o.n;
        if (grid != o.grid) return grid < o.grid;
        if (policy != o.policy) return policy < o.policy;
        return pairs != o.pairs ? pairs < o.pairs : drift < o.drift;
    }
};

}  // namespace

struct mc_system {
    std::vector<Chain> chains;
    mcg::ChainDev *d_chains = nullptr;
    std::vector<mcg::ChainDev> h_chains;
    mcg::Ctl *d_ctl = nullptr;
    mcg::Ctl *h_ctl = nullptr;  // pinned template copied to d_ctl before each launch
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int poisoned = 0;
    int guard_mode = 0;
    long long timeout_ms = 4000;
    int ctas_override = 0;
    long long skip_ticket = -1;
    int use_graph = 1;
    int policy = 0;  // ticket order: 0 group round-robin over chains, 1 sweep-synchronous
    int sm_count = 0, occ = 0;
    int pairs_opt = -1;                 // MC_OPT_PAIRS: -1 automatic, 0 off, 1 on
    int deep_opt = 1;                   // MC_OPT_DEEP_WINDOWS: 1 on (default), 0 off
    long long drift_every = 0;          // MC_OPT_DRIFT_EVERY: accurate energy and drift check every K sweeps (0 off)
    int helpers_opt = 0;                // MC_OPT_HELPERS: 0 off (default), 1 on
    int da_sweeps = 1;                  // MC_OPT_DA_SWEEPS: sweeps per launch of chains with a cell list
    int occ_h = 0;                      // resident CTAs per SM of the helper-warp kernel (0: unavailable)
    int max_clusters = 0;               // resident clusters of two CTAs (0: pairs mode unavailable)
    mcg::PairBox *d_box = nullptr;      // one hand-over box per cluster
    mcg::GuardBoard *d_gb = nullptr;    // the shared guard's board (and its per-chunk sums after it)
    int gb_opt = 1;                     // MC_OPT_SHARED_GUARD
    int da_on = 1;  // chains with a surrogate sweep with delayed acceptance (MC_OPT_DA)
    std::map<std::pair<long long, int>, std::pair<mcg::Ticket *, int>> scheds;  // (n_sweeps, policy) -> schedule
    std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace {

// Host-side validation (Sec. 5.2 hard wall; Sec. 3.3 hard cores): every centre
// within R - sigma/2 and no two closer than sigma, distances in FP64 from the
// FP32 coordinates.  Uniform grid with cell edge >= sigma.
int validate(const float *xyz, int64_t n, double sigma, double R)
{
    const double Rc = R - 0.5 * sigma, Rc2 = Rc * Rc, s2 = sigma * sigma;
    for (int64_t i = 0; i < n; ++i) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        const double r2 = (x * x + y * y) + z * z;
        if (!(r2 <= Rc2)) return fail(MC_ERR_OVERLAP_INIT, "ion %lld lies outside the wall (|r|^2 = %.17g > %.17g)",
                                      (long long)i, r2, Rc2);
    }
    long long m = (long long)std::floor(2.0 * Rc / sigma);
    if (m < 1) m = 1;
    if (m > 600) m = 600;
    const double cell = 2.0 * Rc / (double)m;
    std::vector<long long> head((size_t)(m * m * m), -1), next((size_t)n, -1);
    auto cidx = [&](double v) {
        long long c = (long long)std::floor((v + Rc) / cell);
        return c < 0 ? 0 : (c >= m ? m - 1 : c);
    };
    for (int64_t i = 0; i < n; ++i) {
        const long long cx = cidx(xyz[3 * i]), cy = cidx(xyz[3 * i + 1]), cz = cidx(xyz[3 * i + 2]);
        for (long long ax = cx - 1; ax <= cx + 1; ++ax)
            for (long long ay = cy - 1; ay <= cy + 1; ++ay)
                for (long long az = cz - 1; az <= cz + 1; ++az) {
                    if (ax < 0 || ay < 0 || az < 0 || ax >= m || ay >= m || az >= m) continue;
                    for (long long j = head[(size_t)((ax * m + ay) * m + az)]; j >= 0; j = next[(size_t)j]) {
                        const double dx = (double)xyz[3 * i] - (double)xyz[3 * j];
                        const double dy = (double)xyz[3 * i + 1] - (double)xyz[3 * j + 1];
                        const double dz = (double)xyz[3 * i + 2] - (double)xyz[3 * j + 2];
                        if ((dx * dx + dy * dy) + dz * dz < s2)
                            return fail(MC_ERR_OVERLAP_INIT, "ions %lld and %lld overlap", (long long)j, (long long)i);
                    }
                }
        const size_t c = (size_t)((cx * m + cy) * m + cz);
        next[(size_t)i] = head[c];
        head[c] = i;
    }
    return MC_OK;
}

// Positions become the state after sweep c.sweeps - 1 (buffer c.sweeps & 1);
// the padding slots of both buffers hold far-away ions of valence 0.
int upload_positions(mc_system *h, Chain &c, const float *xyz, cudaStream_t st)
{
    std::vector<float4> buf((size_t)c.B * mcg::S);
    for (int i = 0; i < c.N; ++i) buf[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], c.q[i]);
    for (size_t i = c.N; i < buf.size(); ++i) buf[i] = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
    CK(cudaMemcpyAsync(c.cur(), buf.data(), sizeof(float4) * buf.size(), cudaMemcpyHostToDevice, st));
    if (c.B * mcg::S > c.N) {
        float4 *other = c.pos[(c.sweeps + 1) & 1];
        CK(cudaMemcpyAsync(other + c.N, buf.data() + c.N, sizeof(float4) * (buf.size() - c.N), cudaMemcpyHostToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    c.sweep_base = c.sweeps;
    (void)h;
    return MC_OK;
}

// Device descriptor of chain c (see mc_device.cuh).
mcg::ChainDev describe(const Chain &c)
{
    mcg::ChainDev d{};
    d.pos[0] = c.pos[0];
    d.pos[1] = c.pos[1];
    d.sweep_base = c.sweep_base;
    d.flags = c.flags;
    d.bits = c.bits;
    d.ledger = c.ledger;
    d.ledger_seq = c.ledger_seq;
    d.stats = c.stats;
    d.sweep = c.sweep;
    d.rec = c.rec;
    d.trace = c.trace;
    d.trace_cap = c.trace_cap;
    d.rec_sweep0 = c.rec_sweep0;
    d.rec_cap = c.rec_cap;
    d.eser = c.eser;
    d.eser_cap = c.eser_cap;
    d.eser_sweep0 = c.eser_sweep0;
    d.N = c.N;
    d.B = c.B;
    d.D = (float)(2.0 * c.h);
    const double s2 = c.sigma * c.sigma;
    d.sig2 = s2;
    // FP32 squared distances carry a relative error below 2^-21; outside
    // s2 (1 -/+ 2^-19) the FP32 comparison already agrees with FP64.
    d.sig2_lo = std::nextafter((float)(s2 * (1.0 - 0x1p-19)), 0.0f);
    d.sig2_hi = std::nextafter((float)(s2 * (1.0 + 0x1p-19)), 3.0e38f);
    double qabs = 0.0;
    for (float v : c.q) qabs += std::fabs((double)v);
    d.a_max = (float)(2.0 * qabs / (c.sigma * (1.0 - 0x1p-17)) * (1.0 + 0x1p-20));
    d.lB = c.lB;
    const double Rc = c.R - 0.5 * c.sigma;
    d.Rc2 = Rc * Rc;
    d.key0 = (unsigned)(c.seed & 0xffffffffu);
    d.key1 = c.chain_id;
    d.ctr3 = (unsigned)(c.seed >> 32);
    d.da = nullptr;
    d.pf = 0u;
    return d;
}

int sync_descriptors(mc_system *h)
{
    h->h_chains.resize(h->chains.size());
    for (size_t i = 0; i < h->chains.size(); ++i) {
        h->h_chains[i] = describe(h->chains[i]);
        if (h->chains[i].da && h->da_on) {
            h->h_chains[i].da = h->chains[i].dda;
            h->h_chains[i].pf = h->chains[i].pf ? 1u : 0u;
        }
    }
    CK(cudaMemcpy(h->d_chains, h->h_chains.data(), sizeof(mcg::ChainDev) * h->h_chains.size(), cudaMemcpyHostToDevice));
    return MC_OK;
}

// The checks of mc_create on one chain description: parameters, finite inputs, wall and overlap.
int check_desc(const mc_chain_desc &d)
{
    if (!d.pos_xyz || !d.q) return fail(MC_ERR_INVALID, "NULL positions or valences");
    if (d.n < 1 || d.n > (int64_t)1 << 30) return fail(MC_ERR_INVALID, "N = %lld out of range", (long long)d.n);
    if (!(d.sigma > 0.0) || !(d.l_B >= 0.0) || !(d.R > 0.5 * d.sigma) || !(d.half_width >= 0.0) ||
        !std::isfinite(d.l_B) || !std::isfinite(d.R) || !std::isfinite(d.half_width))
        return fail(MC_ERR_INVALID, "invalid parameters (sigma %g, l_B %g, R %g, h %g)", d.sigma, d.l_B, d.R,
                    d.half_width);
    for (int64_t i = 0; i < d.n; ++i)
        if (!std::isfinite(d.q[i]) || !std::isfinite(d.pos_xyz[3 * i]) || !std::isfinite(d.pos_xyz[3 * i + 1]) ||
            !std::isfinite(d.pos_xyz[3 * i + 2]))
            return fail(MC_ERR_INVALID, "non-finite input at ion %lld", (long long)i);
    return validate(d.pos_xyz, d.n, d.sigma, d.R);
}

int init_chain(mc_system *h, Chain &c, const mc_chain_desc &d)
{
    int rc = check_desc(d);
    if (rc) return rc;
    c.N = (int)d.n;
    c.B = (c.N + mcg::S - 1) / mcg::S;
    c.sigma = d.sigma;
    c.lB = d.l_B;
    c.R = d.R;
    c.h = d.half_width;
    c.seed = d.seed;
    c.chain_id = d.chain_id;
    c.q.assign(d.q, d.q + d.n);
    CK(cudaMalloc(&c.pos[0], sizeof(float4) * (size_t)c.B * mcg::S));
    CK(cudaMalloc(&c.pos[1], sizeof(float4) * (size_t)c.B * mcg::S));
    CK(cudaMalloc(&c.flags, sizeof(unsigned long long) * (size_t)c.B * mcg::WORDS));
    CK(cudaMalloc(&c.bits, sizeof(unsigned long long) * (size_t)c.B * mcg::WORDS));
    CK(cudaMalloc(&c.slab, 64 + 8 * mcg::NCOUNTERS));
    CK(cudaMemsetAsync(c.flags, 0, sizeof(unsigned long long) * (size_t)c.B * mcg::WORDS, h->stream));
    CK(cudaMemsetAsync(c.bits, 0, sizeof(unsigned long long) * (size_t)c.B * mcg::WORDS, h->stream));
    CK(cudaMemsetAsync(c.slab, 0, 64 + 8 * mcg::NCOUNTERS, h->stream));
    c.ledger = (double *)c.slab;
    c.ledger_seq = (unsigned long long *)(c.slab + 8);
    c.sweep = (unsigned long long *)(c.slab + 16);
    c.e_out = (double *)(c.slab + 24);
    c.drift = (double *)(c.slab + 32);  // 3 doubles: last drift, maximum, checks
    c.stats = (unsigned long long *)(c.slab + 64);  // NCOUNTERS counters
    rc = upload_positions(h, c, d.pos_xyz, h->stream);
    if (rc) return rc;
    CK(cudaMalloc(&c.eparts, sizeof(double) * (size_t)mcg_host::energy_ff_parts(c.N)));
    CK(mcg_host::energy_ff_launch(c.cur(), nullptr, nullptr, c.N, c.lB, c.eparts, c.ledger, nullptr, nullptr, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

void free_chain(Chain &c)
{
    cudaFree(c.pos[0]);
    cudaFree(c.pos[1]);
    cudaFree(c.d_xyz);
    cudaFree(c.d_vcnt);
    cudaFree(c.d_vids);
    cudaFree(c.d_verr);
    cudaFree(c.flags);
    cudaFree(c.bits);
    cudaFree(c.slab);
    cudaFree(c.eparts);
    cudaFree(c.rec);
    cudaFree(c.trace);
    cudaFree(c.eser);
    cudaFree(c.dda);
    cudaFree(c.d_w);
    cudaFree(c.d_w2n);
    cudaFree(c.d_cell_start);
    cudaFree(c.d_cell_ions);
    cudaFree(c.d_slot_of);
    cudaFree(c.d_cnt);
    cudaFree(c.d_cellid);
    cudaFree(c.d_fill);
    cudaFree(c.d_cell_pos);
    c = Chain();
}

int check(mc_system *h)
{
    if (!h) return fail(MC_ERR_INVALID, "NULL handle");
    if (h->poisoned) return fail(MC_ERR_POISONED, "handle poisoned by an earlier device error: %s", g_err.c_str());
    return MC_OK;
}

int check_chain(mc_system *h, int chain)
{
    int rc = check(h);
    if (rc) return rc;
    if (chain < 0 || chain >= (int)h->chains.size()) return fail(MC_ERR_INVALID, "chain %d out of range", chain);
    return MC_OK;
}

void write_ctl(mc_system *h);

int create_common(const mc_chain_desc *descs, int n_chains, mc_handle *out)
{
    if (!out || !descs || n_chains < 1) return fail(MC_ERR_INVALID, "bad arguments to mc_create_batch");
    *out = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    mc_system *h = new mc_system();
    auto bail = [&](int rc) {
        for (auto &c : h->chains) free_chain(c);
        cudaFree(h->d_chains);
        cudaFree(h->d_ctl);
        cudaFree(h->d_gb);
        cudaFree(h->d_box);
        if (h->h_ctl) cudaFreeHost(h->h_ctl);
        if (h->own_stream) cudaStreamDestroy(h->own_stream);
        delete h;
        return rc;
    };
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(MC_ERR_CUDA, "cudaStreamCreate failed"));
    h->stream = h->own_stream;
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        mcg_host::sweep_configure() != cudaSuccess || mcg_host::sweep_occupancy(&h->occ) != cudaSuccess)
        return bail(fail(MC_ERR_CUDA, "kernel configuration failed: %s", cudaGetErrorString(cudaGetLastError())));
    if (mcg_host::sweep_occupancy_h(&h->occ_h) != cudaSuccess) {
        h->occ_h = 0;  // the helper-warp kernel cannot run: one group of warps per work item
        cudaGetLastError();
    }
    if (mcg_host::sweep_max_clusters(&h->max_clusters) != cudaSuccess) {
        h->max_clusters = 0;  // clusters unavailable: pairs mode stays off
        cudaGetLastError();
    }
    if (h->occ < 1) return bail(fail(MC_ERR_CUDA, "sweep kernel does not fit on an SM"));
    h->chains.resize(n_chains);
    for (int i = 0; i < n_chains; ++i) {
        int rc = init_chain(h, h->chains[i], descs[i]);
        if (rc) {
            std::string msg = g_err;
            bail(rc);
            g_err = "chain " + std::to_string(i) + ": " + msg;
            return rc;
        }
    }
    if (cudaMalloc(&h->d_chains, sizeof(mcg::ChainDev) * n_chains) != cudaSuccess ||
        cudaMalloc(&h->d_ctl, sizeof(mcg::Ctl)) != cudaSuccess ||
        cudaMallocHost(&h->h_ctl, sizeof(mcg::Ctl)) != cudaSuccess ||
        cudaMalloc(&h->d_box, sizeof(mcg::PairBox) * (size_t)std::max(1, h->sm_count)) != cudaSuccess)
        return bail(fail(MC_ERR_OOM, "allocation of launch state failed"));
    {
        // the shared guard's board: the request, then the sums of every chunk of the largest chain
        long long nmax = 1;
        for (const auto &c : h->chains) nmax = std::max(nmax, ((long long)c.N + mcg::GB_CHUNK - 1) / mcg::GB_CHUNK);
        if (nmax <= 0xffff) {
            const size_t off = (sizeof(mcg::GuardBoard) + 255) & ~(size_t)255;
            char *p = nullptr;
            if (cudaMalloc(&p, off + 2 * sizeof(double) * (size_t)nmax) != cudaSuccess)
                return bail(fail(MC_ERR_OOM, "allocation of the guard board failed"));
            h->d_gb = reinterpret_cast<mcg::GuardBoard *>(p);
            mcg::GuardBoard gb{};
            gb.part = reinterpret_cast<double *>(p + off);
            gb.bpart = gb.part + nmax;
            if (cudaMemcpy(h->d_gb, &gb, sizeof gb, cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(MC_ERR_CUDA, "guard board setup failed"));
        }
    }
    int rc = sync_descriptors(h);
    if (rc) return bail(rc);
    write_ctl(h);
    *out = h;
    return MC_OK;
}

// Work items of n sweeps for all chains: chain-interleaved, each chain's
// groups in stream order (sweep-major, group-minor).
int schedule_for(mc_system *h, long long n, mcg::Ticket **d, int *count)
{
    auto it = h->scheds.find({n, h->policy});
    if (it != h->scheds.end()) {
        *d = it->second.first;
        *count = it->second.second;
        return MC_OK;
    }
    std::vector<mcg::Ticket> t;
    long long total = 0, longest = 0;
    for (auto &c : h->chains) {
        total += (long long)c.B * n;
        longest = std::max(longest, (long long)c.B * n);
    }
    if (total > (1ll << 31) - 1) return fail(MC_ERR_INVALID, "too many work items (%lld); sweep in smaller batches", total);
    t.reserve((size_t)total);
    if (h->policy == 0) {
        // one group of every chain in turn: every chain advances at the same rate in groups
        for (long long step = 0; step < longest; ++step)
            for (size_t ci = 0; ci < h->chains.size(); ++ci) {
                const Chain &c = h->chains[ci];
                if (step < (long long)c.B * n)
                    t.push_back(mcg::Ticket{(int)ci, (int)(step % c.B), (int)(step / c.B), 0});
            }
    } else {
        // sweep-synchronous: all chains' sweep s before sweep s + 1, groups interleaved within a sweep, so
        // large chains (more groups per sweep) get proportionally more work items early
        int maxB = 0;
        for (auto &c : h->chains) maxB = std::max(maxB, c.B);
        for (long long sw = 0; sw < n; ++sw)
            for (int g = 0; g < maxB; ++g)
                for (size_t ci = 0; ci < h->chains.size(); ++ci)
                    if (g < h->chains[ci].B) t.push_back(mcg::Ticket{(int)ci, g, (int)sw, 0});
    }
    mcg::Ticket *dp = nullptr;
    CK(cudaMalloc(&dp, sizeof(mcg::Ticket) * t.size()));
    CK(cudaMemcpy(dp, t.data(), sizeof(mcg::Ticket) * t.size(), cudaMemcpyHostToDevice));
    h->scheds[{n, h->policy}] = {dp, (int)t.size()};
    *d = dp;
    *count = (int)t.size();
    return MC_OK;
}

// Work items of a launch of n sweeps: the groups of every chain, n times.  Items of the next sweep may be in
// flight with the current sweep's: each waits for its group's previous version, and a group's new version
// overwrites the buffer of the version before its previous one only after every item of the previous sweep
// has published (chain order), so no reader of that buffer remains.
int grid_for(mc_system *h, long long n_sweeps = 1)
{
    long long useful = 0;
    for (auto &c : h->chains) useful += c.B;
    long long g = (long long)h->sm_count * h->occ;
    if (h->ctas_override > 0) g = std::min<long long>(g, h->ctas_override);
    g = std::min(g, useful * std::max(1LL, n_sweeps));
    // delayed acceptance: fewer resident CTAs than the exclusion depth, so every counted ion's group has
    // finished when a work item starts
    if (h->da_on)
        for (auto &c : h->chains)
            if (c.da) g = std::min<long long>(g, c.hda.W - 1);
    return (int)std::max<long long>(1, g);
}

// Captured sweep graphs depend on which chains sweep with delayed acceptance.
void drop_graphs(mc_system *h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    h->graphs.clear();
}

bool any_da(const mc_system *h)
{
    if (!h->da_on) return false;
    for (auto &c : h->chains)
        if (c.da) return true;
    return false;
}

// Helper warps (MC_OPT_HELPERS): the 2T-thread kernel whose second half takes half of every tile pass; used when
// asked for (directly or by the autotuner) and pairs mode is off.  Off by default: on GB300 it measured slower.
bool pairs_on(const mc_system *h);
bool helpers_on(const mc_system *h)
{
    if (h->occ_h < 1 || h->helpers_opt != 1) return false;
    return !pairs_on(h);
}

// The periodic drift check (MC_OPT_DRIFT_EVERY): the accurate energy of every chain's current positions (the
// buffer is chosen on the device from the sweep counter, so captured graphs replay correctly) and the drift
// |ledger - E| folded into the chain's last / maximum / count.
cudaError_t enqueue_drift(mc_system *h)
{
    cudaError_t e = cudaSuccess;
    for (size_t ci = 0; ci < h->chains.size() && e == cudaSuccess; ++ci) {
        Chain &c = h->chains[ci];
        e = mcg_host::energy_ff_launch(c.pos[0], c.pos[1], c.sweep, c.N, c.lB, c.eparts, c.e_out, c.ledger, c.drift,
                                       h->stream);
    }
    return e;
}

// Chains with a cell list (delayed acceptance, the overlap prefilter): launches of at most MC_OPT_DA_SWEEPS sweeps,
// each preceded by the preparation of every such chain's cell list from the launch's start positions, and cut at
// the drift check's period.  The control block is copied once; later launches only reset its ticket counter, so an
// error or abort stays visible.
cudaError_t enqueue_da(mc_system *h, long long n, int grid)
{
    cudaError_t e = cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(mcg::Ctl), cudaMemcpyHostToDevice, h->stream);
    for (long long done = 0; done < n && e == cudaSuccess;) {
        long long m = std::min<long long>(h->da_sweeps, n - done);
        if (h->drift_every > 0) m = std::min(m, h->drift_every - done % h->drift_every);
        mcg::Ticket *sched = nullptr;
        int count = 0;
        if (schedule_for(h, m, &sched, &count) != MC_OK) return cudaErrorInvalidValue;
        if (done > 0) e = cudaMemsetAsync(&h->d_ctl->ticket, 0, sizeof(unsigned), h->stream);
        for (size_t ci = 0; ci < h->chains.size(); ++ci) {
            Chain &c = h->chains[ci];
            if (!c.da || e != cudaSuccess) continue;
            e = c.pf ? mcg_host::da_prep_bucket_launch(h->d_chains + ci, c.N, c.dda, c.ncell, c.d_cnt, c.d_cell_pos,
                                                       c.d_slot_of, h->stream)
                     : mcg_host::da_prep_launch(h->d_chains + ci, c.N, c.dda, c.ncell, c.d_cnt, c.d_cellid,
                                                c.d_cell_start, c.d_fill, c.d_cell_ions, c.d_cell_pos, c.d_slot_of,
                                                h->stream);
        }
        if (e == cudaSuccess)
            e = mcg_host::sweep_launch(grid, h->d_chains, sched, count, h->d_ctl, (int)h->chains.size(), m, h->stream,
                                       false, helpers_on(h), true);
        done += m;
        if (e == cudaSuccess && h->drift_every > 0 && done % h->drift_every == 0) e = enqueue_drift(h);
    }
    return e;
}

// Plain chains: n sweeps as persistent launches of at most K sweeps each (K = MC_OPT_DRIFT_EVERY, or all n when the
// check is off), a drift check after every full K.
cudaError_t enqueue_plain(mc_system *h, long long n, int grid, bool pr)
{
    const int nch = (int)h->chains.size();
    const long long K = h->drift_every > 0 ? h->drift_every : n;
    cudaError_t e = cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(mcg::Ctl), cudaMemcpyHostToDevice, h->stream);
    for (long long done = 0; done < n && e == cudaSuccess;) {
        const long long m = std::min(K, n - done);
        mcg::Ticket *sched = nullptr;
        int count = 0;
        if (schedule_for(h, m, &sched, &count) != MC_OK) return cudaErrorInvalidValue;
        if (done > 0) e = cudaMemsetAsync(&h->d_ctl->ticket, 0, sizeof(unsigned), h->stream);
        if (e == cudaSuccess)
            e = mcg_host::sweep_launch(grid, h->d_chains, sched, count, h->d_ctl, nch, m, h->stream, pr, !pr && helpers_on(h),
                                       false);
        done += m;
        if (e == cudaSuccess && h->drift_every > 0 && m == K) e = enqueue_drift(h);
    }
    return e;
}

int enqueue_sweeps(mc_system *h, long long n)
{
    mcg::Ticket *sched = nullptr;
    int count = 0;
    const bool da = any_da(h);
    const long long per = da ? std::min<long long>(n, h->da_sweeps)
                             : (h->drift_every > 0 ? std::min<long long>(n, h->drift_every) : n);
    int rc = schedule_for(h, per, &sched, &count);
    if (rc) return rc;
    if (da) {  // every launch length enqueue_da will use, before any capture (schedules are allocated once)
        long long seen[4] = {per, 0, 0, 0};
        int ns = 1;
        for (long long done = 0; done < n;) {
            long long m = std::min<long long>(h->da_sweeps, n - done);
            if (h->drift_every > 0) m = std::min(m, h->drift_every - done % h->drift_every);
            bool have = false;
            for (int q = 0; q < ns; ++q) have |= seen[q] == m;
            if (!have) {
                mcg::Ticket *s2 = nullptr;
                int c2 = 0;
                if ((rc = schedule_for(h, m, &s2, &c2))) return rc;
                if (ns < 4) seen[ns++] = m;
            }
            done += m;
        }
    }
    if (!da && h->drift_every > 0 && n > h->drift_every) {  // the schedule of the last, shorter launch
        mcg::Ticket *s2 = nullptr;
        int c2 = 0;
        if ((rc = schedule_for(h, n % h->drift_every ? n % h->drift_every : h->drift_every, &s2, &c2))) return rc;
    }
    const bool pr = !da && h->h_ctl->pairs != 0;
    int grid = grid_for(h, per);
    if (pr) grid = std::max(2, std::min(grid & ~1, 2 * h->max_clusters));  // whole clusters of two
    const int nch = (int)h->chains.size();
    if (h->use_graph) {
        GraphKey key{n, grid, h->policy, pr ? 1 : 0, h->drift_every};
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = cudaSuccess, e2 = cudaSuccess;
            if (da) {
                e2 = enqueue_da(h, n, grid);
            } else {
                e2 = enqueue_plain(h, n, grid, pr);
            }
            cudaError_t e3 = cudaStreamEndCapture(h->stream, &g);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return fail(MC_ERR_CUDA, "graph capture failed: %s / %s / %s", cudaGetErrorString(e1),
                            cudaGetErrorString(e2), cudaGetErrorString(e3));
            }
            cudaGraphExec_t ge = nullptr;
            cudaError_t e4 = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e4 != cudaSuccess) return fail(MC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e4));
            it = h->graphs.emplace(key, ge).first;
        }
        CK(cudaGraphLaunch(it->second, h->stream));
    } else if (da) {
        CK(enqueue_da(h, n, grid));
    } else {
        CK(enqueue_plain(h, n, grid, pr));
    }
    for (auto &ch : h->chains) ch.sweeps += (uint64_t)n;
    return MC_OK;
}

// The pinned control block is copied to the device at the start of every
// launch (also inside captured graphs), so it is rewritten only while the
// stream is idle.
// Pairs mode (two CTAs per work item, tiles split) for a single plain chain whose groups fit two waves of SMs
// (at 4 waves, N = 65536, one CTA per item measured 4 % faster), with deep windows on: then every in-flight work item must fold each newly published tile as it appears,
// and splitting the tiles halves that latency.  Without deep windows the chain waits on the tile two groups
// back and one CTA per item (twice as many in flight) measured faster.  Chains with delayed acceptance and
// batches run one CTA per work item.
bool pairs_on(const mc_system *h)
{
    if (h->max_clusters < 1 || any_da(h) || h->pairs_opt == 0) return false;
    if (h->pairs_opt == 1) return true;
    return h->deep_opt && h->chains.size() == 1 && h->chains[0].B <= 2LL * h->sm_count;
}

void write_ctl(mc_system *h)
{
    mcg::Ctl *c = h->h_ctl;
    std::memset(c, 0, sizeof(mcg::Ctl));
    c->guard_mode = h->guard_mode;
    c->timeout_ns = h->timeout_ms * 1000000ll;
    c->skip_ticket = h->skip_ticket;
    c->pairs = pairs_on(h) ? 1 : 0;
    c->deep = h->deep_opt;
    c->box = h->d_box;
    c->gb = h->gb_opt ? h->d_gb : nullptr;
}

int finish(mc_system *h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->poisoned = 1;
        return fail(MC_ERR_CUDA, "sweep failed: %s", cudaGetErrorString(e));
    }
    mcg::Ctl c;
    e = cudaMemcpy(&c, h->d_ctl, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        h->poisoned = 1;
        return fail(MC_ERR_CUDA, "reading sweep status failed: %s", cudaGetErrorString(e));
    }
    if (c.err) {
        h->poisoned = 1;
        if (c.err == mcg::KERR_TIMEOUT)
            return fail(MC_ERR_TIMEOUT, "a device-side wait expired after %lld ms (group %u, sweep tag %u)",
                        h->timeout_ms, (unsigned)(c.err_info >> 32), (unsigned)c.err_info);
        return fail(MC_ERR_CUDA, "inter-CTA protocol violation (code %d)", c.err);
    }
    return MC_OK;
}

}  // namespace

namespace mcg_host {
int set_error(int code, const char *msg)
{
    return fail(code, "%s", msg);
}
}  // namespace mcg_host

extern "C" {

int mc_create(const float *pos_xyz, const float *q, int64_t n, double sigma, double l_B, double R, double half_width,
              uint64_t seed, uint32_t chain_id, mc_handle *out)
{
    mc_chain_desc d{pos_xyz, q, n, sigma, l_B, R, half_width, seed, chain_id};
    return create_common(&d, 1, out);
}

int mc_create_batch(const mc_chain_desc *descs, int n_chains, mc_handle *out)
{
    Range nv("mc_create_batch");
    return create_common(descs, n_chains, out);
}

int mc_sweep_async(mc_handle h, int64_t n_sweeps)
{
    Range nv("mc_sweep_async");
    int rc = check(h);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(MC_ERR_INVALID, "n_sweeps < 0");
    if (n_sweeps == 0) return MC_OK;
    return enqueue_sweeps(h, n_sweeps);
}

int mc_synchronize(mc_handle h)
{
    Range nv("mc_synchronize");
    int rc = check(h);
    if (rc) return rc;
    return finish(h);
}

int mc_sweep(mc_handle h, int64_t n_sweeps)
{
    Range nv("mc_sweep");
    int rc = mc_sweep_async(h, n_sweeps);
    if (rc) return rc;
    return finish(h);
}

int mc_set_stream(mc_handle h, void *cuda_stream)
{
    int rc = check(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    return MC_OK;
}

int mc_energy(mc_handle h, int chain, double *ledger, double *recomputed)
{
    Range nv("mc_energy");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    if (ledger) CK(cudaMemcpy(ledger, c.ledger, sizeof(double), cudaMemcpyDeviceToHost));
    if (recomputed) {
        CK(mcg_host::energy_ff_launch(c.cur(), nullptr, nullptr, c.N, c.lB, c.eparts, c.e_out, nullptr, nullptr,
                                      h->stream));
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaMemcpy(recomputed, c.e_out, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return MC_OK;
}

int mc_gr_histogram(mc_handle h, int chain, int n_bins, double r_max, double wall_margin, uint64_t *counts)
{
    Range nv("mc_gr_histogram");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (n_bins < 1 || n_bins > 4096 || !(r_max > 0.0) || !counts || !std::isfinite(wall_margin))
        return fail(MC_ERR_INVALID, "bad histogram arguments");
    Chain &c = h->chains[chain];
    const double dr = r_max / (double)n_bins;
    const double Rc = c.R - 0.5 * c.sigma;
    const double lim = Rc - wall_margin;
    const double lim2 = lim * lim;
    std::vector<unsigned long long> hc((size_t)3 * n_bins, 0ull);
    if (wall_margin > 0.0 && lim < 0.0) return MC_OK;  // no interior ions
    unsigned long long *d = nullptr;
    CK(cudaMalloc(&d, sizeof(unsigned long long) * hc.size()));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * hc.size(), h->stream);
    const float hi = std::nextafter((float)(r_max * r_max * (1.0 + 0x1p-18)), 3.0e38f);
    if (e == cudaSuccess) e = mcg_host::gr_launch(c.cur(), c.N, n_bins, dr, hi, wall_margin > 0.0 ? 1 : 0, lim2, d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), d, sizeof(unsigned long long) * hc.size(), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "histogram: %s", cudaGetErrorString(e));
    for (size_t i = 0; i < hc.size(); ++i) counts[i] += hc[i];
    return MC_OK;
}

// Device staging of host positions and the grid of their check (allocated on first use, kept with the chain).
static int ensure_pos_scratch(Chain &c)
{
    if (c.d_xyz) return MC_OK;
    const double Rc = c.R - 0.5 * c.sigma;
    // cells of edge >= sigma, at most 4 per ion and 600 per axis; cap = k^3 sub-cubes of diagonal below sigma
    long long m = (long long)std::floor(2.0 * Rc / c.sigma);
    m = std::min(m, std::min(600LL, (long long)std::cbrt(4.0 * (double)c.N) + 1));
    m = std::max(1LL, m);
    const double edge = 2.0 * Rc / (double)m;
    const int k = (int)std::floor(edge * std::sqrt(3.0) / c.sigma * (1.0 + 1e-9)) + 1;
    c.vm = (int)m;
    c.vcap = std::min(1000, k * k * k);
    CK(cudaMalloc(&c.d_xyz, sizeof(float) * 3 * (size_t)c.N));
    CK(cudaMalloc(&c.d_vcnt, sizeof(int) * (size_t)(m * m * m)));
    CK(cudaMalloc(&c.d_vids, sizeof(int) * (size_t)(m * m * m) * (size_t)c.vcap));
    CK(cudaMalloc(&c.d_verr, sizeof(unsigned long long)));
    return MC_OK;
}

int mc_get_positions(mc_handle h, int chain, float *pos_xyz)
{
    Range nv("mc_get_positions");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!pos_xyz) return fail(MC_ERR_INVALID, "NULL buffer");
    Chain &c = h->chains[chain];
    if ((rc = ensure_pos_scratch(c))) return rc;
    CK(mcg_host::pos_unpack_launch(c.cur(), c.N, c.d_xyz, h->stream));
    CK(cudaMemcpyAsync(pos_xyz, c.d_xyz, sizeof(float) * 3 * (size_t)c.N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

// The positions are copied to the device, checked there by the validation rule (FP64, every pair within sigma
// through a bucket grid) and packed into the current buffer only if they pass; the valences stay.
int mc_set_positions(mc_handle h, int chain, const float *pos_xyz)
{
    Range nv("mc_set_positions");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!pos_xyz) return fail(MC_ERR_INVALID, "NULL buffer");
    Chain &c = h->chains[chain];
    if ((rc = ensure_pos_scratch(c))) return rc;
    const double Rc = c.R - 0.5 * c.sigma;
    CK(cudaMemcpyAsync(c.d_xyz, pos_xyz, sizeof(float) * 3 * (size_t)c.N, cudaMemcpyHostToDevice, h->stream));
    CK(mcg_host::pos_check_launch(c.d_xyz, c.N, Rc, 2.0 * Rc / (double)c.vm, c.vm, c.vcap, c.sigma * c.sigma,
                                  c.d_vcnt, c.d_vids, c.d_verr, h->stream));
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, c.d_verr, sizeof key, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (key != ~0ull) {
        const unsigned kind = (unsigned)(key >> 62);
        if (kind == 1) return fail(MC_ERR_OVERLAP_INIT, "ion %lld lies outside the wall", (long long)(key & 0x7fffffffull));
        if (kind == 2)
            return fail(MC_ERR_OVERLAP_INIT, "ions %lld and %lld overlap", (long long)(key & 0x7fffffffull),
                        (long long)((key >> 31) & 0x7fffffffull));
        return fail(MC_ERR_OVERLAP_INIT, "ions overlap (more than %d in a cell of edge %.6g)", c.vcap, 2.0 * Rc / c.vm);
    }
    CK(mcg_host::pos_pack_launch(c.d_xyz, c.N, c.cur(), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    c.sweep_base = c.sweeps;
    return sync_descriptors(h);
}

int mc_stats(mc_handle h, int chain, mc_stats_t *out)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!out) return fail(MC_ERR_INVALID, "NULL output");
    Chain &c = h->chains[chain];
    unsigned long long v[mcg::NCOUNTERS];
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(v, c.stats, sizeof v, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof *out);
    out->sweeps = c.sweeps;
    out->accepts = v[mcg::CNT_ACCEPT];
    out->rej_metropolis = v[mcg::CNT_METRO];
    out->rej_overlap = v[mcg::CNT_OVERLAP];
    out->rej_wall = v[mcg::CNT_WALL];
    out->guard_fp64 = v[mcg::CNT_FP64];
    out->decided_interval = v[mcg::CNT_INTERVAL];
    out->tier2 = v[mcg::CNT_T2];
    out->tier3 = v[mcg::CNT_T3];
    out->tier4 = v[mcg::CNT_T4];
    out->rounds = v[mcg::CNT_ROUNDS];
    out->cyc_wait_window = v[mcg::CNT_CYC_WIN];
    out->cyc_tiles = v[mcg::CNT_CYC_TILES];
    out->cyc_resolve = v[mcg::CNT_CYC_RESOLVE];
    out->cyc_guard = v[mcg::CNT_CYC_GUARD];
    out->cyc_total = v[mcg::CNT_CYC_TOTAL];
    out->cyc_tier[0] = v[mcg::CNT_CYC_T2];
    out->cyc_tier[1] = v[mcg::CNT_CYC_T3];
    out->cyc_tier[2] = v[mcg::CNT_CYC_T4];
    out->ovl_scan = v[mcg::CNT_OVL_SCAN];
    out->cyc_ovl_scan = v[mcg::CNT_CYC_OVL];
    out->da_rej1 = v[mcg::CNT_DA_REJ1];
    out->da_ovl1 = v[mcg::CNT_DA_OVL1];
    out->da_fp64 = v[mcg::CNT_DA_FP64];
    out->cyc_da1 = v[mcg::CNT_CYC_DA1];
    for (int q = 0; q < 4; ++q) out->cyc_da_part[q] = v[mcg::CNT_CYC_DA_PART + q];
    double dr[3];
    CK(cudaMemcpy(dr, c.drift, sizeof dr, cudaMemcpyDeviceToHost));
    out->drift_checks = (uint64_t)dr[2];
    out->drift_last = dr[0];
    out->drift_max = dr[1];
    return MC_OK;
}

int mc_get_state(mc_handle h, int chain, float *pos_xyz, uint64_t *sweeps, double *ledger, mc_stats_t *stats)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (pos_xyz && (rc = mc_get_positions(h, chain, pos_xyz))) return rc;
    if (sweeps) *sweeps = h->chains[chain].sweeps;
    if (ledger && (rc = mc_energy(h, chain, ledger, nullptr))) return rc;
    if (stats && (rc = mc_stats(h, chain, stats))) return rc;
    return MC_OK;
}

int mc_set_state(mc_handle h, int chain, const float *pos_xyz, uint64_t sweeps, double ledger, const mc_stats_t *stats)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    Chain &c = h->chains[chain];
    if (sweeps >= 0xfffffff0ull) return fail(MC_ERR_INVALID, "sweep count too large");
    if (pos_xyz && (rc = validate(pos_xyz, c.N, c.sigma, c.R))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    if (!pos_xyz && ((c.sweeps ^ sweeps) & 1))  // keep the current positions in the buffer of the new parity
        CK(cudaMemcpy(c.pos[sweeps & 1], c.cur(), sizeof(float4) * (size_t)c.B * mcg::S, cudaMemcpyDeviceToDevice));
    c.sweeps = sweeps;
    if (pos_xyz) {
        rc = upload_positions(h, c, pos_xyz, h->stream);
        if (rc) return rc;
    } else {
        c.sweep_base = sweeps;
    }
    std::vector<unsigned long long> fl((size_t)c.B * mcg::WORDS, (unsigned long long)(unsigned)sweeps << 32);
    CK(cudaMemcpy(c.flags, fl.data(), sizeof(unsigned long long) * fl.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.bits, fl.data(), sizeof(unsigned long long) * fl.size(), cudaMemcpyHostToDevice));
    unsigned long long seq = (unsigned long long)sweeps * (unsigned long long)c.B;
    unsigned long long sw = sweeps;
    CK(cudaMemcpy(c.ledger, &ledger, sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.ledger_seq, &seq, sizeof seq, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.sweep, &sw, sizeof sw, cudaMemcpyHostToDevice));
    if (stats) {
        unsigned long long v[mcg::NCOUNTERS] = {};
        v[mcg::CNT_ACCEPT] = stats->accepts;
        v[mcg::CNT_METRO] = stats->rej_metropolis;
        v[mcg::CNT_OVERLAP] = stats->rej_overlap;
        v[mcg::CNT_WALL] = stats->rej_wall;
        v[mcg::CNT_FP64] = stats->guard_fp64;
        v[mcg::CNT_INTERVAL] = stats->decided_interval;
        v[mcg::CNT_T2] = stats->tier2;
        v[mcg::CNT_T3] = stats->tier3;
        v[mcg::CNT_T4] = stats->tier4;
        CK(cudaMemcpy(c.stats, v, sizeof v, cudaMemcpyHostToDevice));
    }
    c.sweeps = sweeps;
    if (c.rec) c.rec_sweep0 = sweeps;
    return sync_descriptors(h);
}

int mc_num_chains(mc_handle h)
{
    int rc = check(h);
    return rc ? rc : (int)h->chains.size();
}

int64_t mc_num_ions(mc_handle h, int chain)
{
    int rc = check_chain(h, chain);
    return rc ? rc : (int64_t)h->chains[chain].N;
}

int mc_record_enable(mc_handle h, int chain, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (cap < 0) return fail(MC_ERR_INVALID, "cap < 0");
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(c.rec);
    c.rec = nullptr;
    c.rec_cap = 0;
    if (cap > 0) {
        CK(cudaMalloc(&c.rec, sizeof(mcg::MoveRec) * (size_t)cap));
        CK(cudaMemset(c.rec, 0xff, sizeof(mcg::MoveRec) * (size_t)cap));
        c.rec_cap = cap;
    }
    c.rec_sweep0 = c.sweeps;
    return sync_descriptors(h);
}

int mc_trace_enable(mc_handle h, int chain, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (cap < 0) return fail(MC_ERR_INVALID, "cap < 0");
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(c.trace);
    c.trace = nullptr;
    c.trace_cap = 0;
    if (cap > 0) {
        CK(cudaMalloc(&c.trace, sizeof(mcg::TraceRec) * (size_t)cap));
        CK(cudaMemset(c.trace, 0, sizeof(mcg::TraceRec) * (size_t)cap));
        c.trace_cap = cap;
    }
    c.rec_sweep0 = c.sweeps;
    return sync_descriptors(h);
}

int64_t mc_trace_read(mc_handle h, int chain, mc_trace_rec *out, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    Chain &c = h->chains[chain];
    if (!out || cap < 0) return fail(MC_ERR_INVALID, "bad trace buffer");
    static_assert(sizeof(mc_trace_rec) == sizeof(mcg::TraceRec), "trace layout");
    const int64_t n = std::min<int64_t>(cap, c.trace_cap);
    CK(cudaStreamSynchronize(h->stream));
    if (n > 0) CK(cudaMemcpy(out, c.trace, sizeof(mc_trace_rec) * (size_t)n, cudaMemcpyDeviceToHost));
    return n;
}

int mc_energy_series_enable(mc_handle h, int chain, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (cap < 0) return fail(MC_ERR_INVALID, "cap < 0");
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(c.eser);
    c.eser = nullptr;
    c.eser_cap = 0;
    if (cap > 0) {
        CK(cudaMalloc(&c.eser, sizeof(double) * (size_t)cap));
        CK(cudaMemset(c.eser, 0xff, sizeof(double) * (size_t)cap));  // NaN until written
        c.eser_cap = cap;
    }
    c.eser_sweep0 = c.sweeps;
    return sync_descriptors(h);
}

int64_t mc_energy_series_read(mc_handle h, int chain, double *out, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!out || cap < 0) return fail(MC_ERR_INVALID, "bad series buffer");
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    const int64_t done = c.sweeps > c.eser_sweep0 ? (int64_t)(c.sweeps - c.eser_sweep0) : 0;
    const int64_t n = std::min<int64_t>(std::min<int64_t>(cap, c.eser_cap), done);
    if (n > 0) CK(cudaMemcpy(out, c.eser, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
    return n;
}

int mc_energy_autocorr(const double *series, int64_t n_series, int64_t n_steps, int64_t stride, int64_t max_lag,
                       double *C, double *Tc)
{
    if (!series || !C) return fail(MC_ERR_INVALID, "NULL series or output");
    if (n_series < 1 || n_steps < 2 || stride < n_steps || max_lag < 0 || max_lag >= n_steps)
        return fail(MC_ERR_INVALID, "bad shape (series %lld, steps %lld, stride %lld, max_lag %lld)",
                    (long long)n_series, (long long)n_steps, (long long)stride, (long long)max_lag);
    // mean over the ensemble and the steps, with a compensated sum (Neumaier) so that the deviations keep their
    // precision when the mean is large against the fluctuations
    double sum = 0.0, comp = 0.0;
    for (int64_t r = 0; r < n_series; ++r)
        for (int64_t k = 0; k < n_steps; ++k) {
            const double v = series[r * stride + k];
            if (!std::isfinite(v)) return fail(MC_ERR_INVALID, "non-finite energy at series %lld step %lld",
                                               (long long)r, (long long)k);
            const double t = sum + v;
            comp += std::fabs(sum) >= std::fabs(v) ? (sum - t) + v : (v - t) + sum;
            sum = t;
        }
    const double mean = (sum + comp) / (double)(n_series * n_steps);
    std::vector<double> dev((size_t)(n_series * n_steps));
    for (int64_t r = 0; r < n_series; ++r)
        for (int64_t k = 0; k < n_steps; ++k) dev[(size_t)(r * n_steps + k)] = series[r * stride + k] - mean;
    for (int64_t n = 0; n <= max_lag; ++n) {
        double acc = 0.0;
        for (int64_t r = 0; r < n_series; ++r) {
            const double *d = &dev[(size_t)(r * n_steps)];
            for (int64_t k = 0; k + n < n_steps; ++k) acc += d[k] * d[k + n];
        }
        C[n] = acc / (double)(n_series * (n_steps - n));
    }
    const double var = C[0];
    if (!(var > 0.0)) return fail(MC_ERR_INVALID, "the energy series has no variance");
    C[0] = 1.0;
    double tc = 0.5;
    for (int64_t n = 1; n <= max_lag; ++n) {
        C[n] /= var;
        tc += C[n];
    }
    if (Tc) *Tc = tc;
    return MC_OK;
}

int mc_dressed_ion_analysis(const uint64_t *counts, int n_bins, double r_max, double n_ref_p, double n_ref_m,
                            double dens_p, double dens_m, double q_p, double q_m, double l_B, double r_lo,
                            double r_hi, double *g, mc_dit_result *out)
{
    if (!counts || !out) return fail(MC_ERR_INVALID, "NULL counts or result");
    if (n_bins < 2 || !(r_max > 0.0) || !(n_ref_p >= 0.0) || !(n_ref_m >= 0.0) || !(dens_p > 0.0) ||
        !(dens_m > 0.0) || !(q_p > 0.0) || !(q_m < 0.0) || !(l_B > 0.0) || !(r_lo < r_hi) || !std::isfinite(r_hi))
        return fail(MC_ERR_INVALID, "bad analysis parameters");
    const double PI = 3.14159265358979323846;
    const double dr = r_max / (double)n_bins;
    std::vector<double> gg((size_t)3 * n_bins);
    for (int k = 0; k < n_bins; ++k) {
        const double r0 = dr * k, r1 = dr * (k + 1);
        const double vb = 4.0 / 3.0 * PI * (r1 * r1 * r1 - r0 * r0 * r0);
        const double norm[3] = {n_ref_p * dens_p * vb, (n_ref_p * dens_m + n_ref_m * dens_p) * vb,
                                n_ref_m * dens_m * vb};
        for (int c = 0; c < 3; ++c)
            gg[(size_t)c * n_bins + k] = norm[c] > 0.0 ? (double)counts[(size_t)c * n_bins + k] / norm[c] : NAN;
    }
    if (g)
        for (size_t t = 0; t < gg.size(); ++t) g[t] = gg[t];
    // usable window bins: all three classes populated, both charge densities screening
    std::vector<double> rr, yp, ym, Upp, Upm, Umm, rhp, rhm;
    for (int k = 0; k < n_bins; ++k) {
        const double r = dr * (k + 0.5);
        if (r < r_lo || r > r_hi) continue;
        const double gpp = gg[k], gpm = gg[(size_t)n_bins + k], gmm = gg[(size_t)2 * n_bins + k];
        if (!(gpp > 0.0 && gpm > 0.0 && gmm > 0.0)) continue;
        const double rho_p = dens_p * q_p * gpp + dens_m * q_m * gpm;  // around a positive ion
        const double rho_m = dens_p * q_p * gpm + dens_m * q_m * gmm;  // around a negative ion
        if (!(rho_p < 0.0 && rho_m > 0.0)) continue;
        rr.push_back(r);
        yp.push_back(std::log(std::fabs(r * rho_p)));
        ym.push_back(std::log(std::fabs(r * rho_m)));
        Upp.push_back(-std::log(gpp));
        Upm.push_back(-std::log(gpm));
        Umm.push_back(-std::log(gmm));
        rhp.push_back(rho_p);
        rhm.push_back(rho_m);
    }
    const size_t nf = rr.size();
    if (nf < 2) return fail(MC_ERR_INVALID, "fewer than 2 usable bins in the window [%g, %g]", r_lo, r_hi);
    // least squares: one slope each, and one common slope with an intercept per line
    double rm = 0.0, ypm = 0.0, ymm = 0.0;
    for (size_t t = 0; t < nf; ++t) {
        rm += rr[t];
        ypm += yp[t];
        ymm += ym[t];
    }
    rm /= (double)nf;
    ypm /= (double)nf;
    ymm /= (double)nf;
    double sxx = 0.0, sxp = 0.0, sxm = 0.0;
    for (size_t t = 0; t < nf; ++t) {
        const double dx = rr[t] - rm;
        sxx += dx * dx;
        sxp += dx * (yp[t] - ypm);
        sxm += dx * (ym[t] - ymm);
    }
    mc_dit_result o{};
    o.kappa = std::sqrt(4.0 * PI * l_B * (dens_p * q_p * q_p + dens_m * q_m * q_m));
    o.kappa_R_pm[0] = -sxp / sxx;
    o.kappa_R_pm[1] = -sxm / sxx;
    o.kappa_R = -(sxp + sxm) / (2.0 * sxx);  // the same abscissae on both lines
    const double k2 = o.kappa_R * o.kappa_R, c4 = 4.0 * PI * l_B;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t t = 0; t < nf; ++t) {
        a[0] += -k2 * Upp[t] / (c4 * rhp[t]);  // q_+^R around a positive ion
        a[1] += -k2 * Upm[t] / (c4 * rhm[t]);  // q_+^R around a negative ion (U_{-+} = U_{+-})
        a[2] += -k2 * Upm[t] / (c4 * rhp[t]);  // q_-^R around a positive ion
        a[3] += -k2 * Umm[t] / (c4 * rhm[t]);  // q_-^R around a negative ion
    }
    o.qR_p[0] = a[0] / (double)nf;
    o.qR_p[1] = a[1] / (double)nf;
    o.qR_m[0] = a[2] / (double)nf;
    o.qR_m[1] = a[3] / (double)nf;
    const double qp = 0.5 * (o.qR_p[0] + o.qR_p[1]), qm = 0.5 * (o.qR_m[0] + o.qR_m[1]);
    double ep = 0.0, em = 0.0;
    for (size_t t = 0; t < nf; ++t) {
        const double e = std::exp(-o.kappa_R * rr[t]) / (4.0 * PI * rr[t]);
        ep += -k2 * qp * e / rhp[t];
        em += -k2 * qm * e / rhm[t];
    }
    o.epsR_pm[0] = ep / (double)nf;
    o.epsR_pm[1] = em / (double)nf;
    o.rd_lhs = k2 / (o.kappa * o.kappa);
    o.rd_rhs = (qp - qm) / (q_p - q_m);
    o.n_fit = (int64_t)nf;
    *out = o;
    return MC_OK;
}

int mc_reduction_run(const mc_chain_desc *desc, int64_t n_sweeps, int scheme, float *pos_out, double *dE_sum,
                     uint64_t *counts, double *ms)
{
    Range nv("mc_reduction_run");
    if (!desc) return fail(MC_ERR_INVALID, "NULL description");
    int rc = check_desc(*desc);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(MC_ERR_INVALID, "n_sweeps < 0");
    if (scheme != MC_SCHEME_SEQUENTIAL && scheme != MC_SCHEME_RANDOM) return fail(MC_ERR_INVALID, "scheme %d", scheme);
    if (!pos_out) return fail(MC_ERR_INVALID, "NULL output positions");
    const mc_chain_desc &d = *desc;
    Chain c;
    c.N = (int)d.n;
    c.B = (c.N + mcg::S - 1) / mcg::S;
    c.sigma = d.sigma;
    c.lB = d.l_B;
    c.R = d.R;
    c.h = d.half_width;
    c.seed = d.seed;
    c.chain_id = d.chain_id;
    c.q.assign(d.q, d.q + d.n);
    const mcg::ChainDev hd = describe(c);  // Philox key, trial width, wall, sigma^2, l_B, N
    // device state, released on every path
    struct Dev {
        mcg::ChainDev *chd = nullptr;
        float4 *pos = nullptr;
        void *part = nullptr;
        unsigned char *slab = nullptr;  // count (u32, padded to 8), sweep (u64), ledger (f64), 5 counters (u64)
        cudaStream_t st = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Dev()
        {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (st) cudaStreamDestroy(st);
            cudaFree(chd);
            cudaFree(pos);
            cudaFree(part);
            cudaFree(slab);
        }
    } v;
    const int N = c.N;
    std::vector<float4> hp((size_t)N);
    for (int i = 0; i < N; ++i)
        hp[(size_t)i] = make_float4(d.pos_xyz[3 * i], d.pos_xyz[3 * i + 1], d.pos_xyz[3 * i + 2], d.q[i]);
    CK(cudaStreamCreateWithFlags(&v.st, cudaStreamNonBlocking));
    CK(cudaMalloc(&v.chd, sizeof(mcg::ChainDev)));
    CK(cudaMalloc(&v.pos, sizeof(float4) * (size_t)N));
    CK(cudaMalloc(&v.part, mcg_host::reduction_part_bytes(N)));
    constexpr size_t SLAB = 8 + 8 + 8 + 5 * 8;
    CK(cudaMalloc(&v.slab, SLAB));
    unsigned *count = reinterpret_cast<unsigned *>(v.slab);
    unsigned long long *sweep = reinterpret_cast<unsigned long long *>(v.slab + 8);
    double *ledger = reinterpret_cast<double *>(v.slab + 16);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(v.slab + 24);
    CK(cudaMemsetAsync(v.slab, 0, SLAB, v.st));
    CK(cudaMemcpyAsync(v.chd, &hd, sizeof hd, cudaMemcpyHostToDevice, v.st));
    CK(cudaMemcpyAsync(v.pos, hp.data(), sizeof(float4) * (size_t)N, cudaMemcpyHostToDevice, v.st));
    CK(cudaEventCreate(&v.e0));
    CK(cudaEventCreate(&v.e1));
    // one sweep = N launches: captured once into a graph for N up to 2^16, plain launches above
    const bool graph = N <= (1 << 16);
    if (graph && n_sweeps > 0) {
        CK(cudaStreamBeginCapture(v.st, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = mcg_host::reduction_sweep_launch(v.chd, v.pos, N, scheme, sweep, v.part, count, ledger, cnt, v.st);
        const cudaError_t ce = cudaStreamEndCapture(v.st, &v.graph);
        CK(le);
        CK(ce);
        CK(cudaGraphInstantiate(&v.exec, v.graph, 0));
    }
    CK(cudaEventRecord(v.e0, v.st));
    for (int64_t s = 0; s < n_sweeps; ++s) {
        if (graph) CK(cudaGraphLaunch(v.exec, v.st));
        else CK(mcg_host::reduction_sweep_launch(v.chd, v.pos, N, scheme, sweep, v.part, count, ledger, cnt, v.st));
    }
    CK(cudaEventRecord(v.e1, v.st));
    CK(cudaStreamSynchronize(v.st));
    if (ms) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, v.e0, v.e1));
        *ms = (double)t;
    }
    CK(cudaMemcpy(hp.data(), v.pos, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToHost));
    for (int i = 0; i < N; ++i) {
        pos_out[3 * i] = hp[(size_t)i].x;
        pos_out[3 * i + 1] = hp[(size_t)i].y;
        pos_out[3 * i + 2] = hp[(size_t)i].z;
    }
    double led = 0.0;
    unsigned long long hc[5];
    CK(cudaMemcpy(&led, ledger, sizeof led, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost));
    if (dE_sum) *dE_sum = led;
    if (counts)
        for (int q = 0; q < 5; ++q) counts[q] = hc[q];
    return MC_OK;
}

int64_t mc_record_read(mc_handle h, int chain, mc_record *out, int64_t cap)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    Chain &c = h->chains[chain];
    if (!out || cap < 0) return fail(MC_ERR_INVALID, "bad record buffer");
    const int64_t n = std::min<int64_t>(cap, c.rec_cap);
    static_assert(sizeof(mc_record) == sizeof(mcg::MoveRec), "record layout");
    CK(cudaStreamSynchronize(h->stream));
    if (n > 0) CK(cudaMemcpy(out, c.rec, sizeof(mc_record) * (size_t)n, cudaMemcpyDeviceToHost));
    return n;
}

static int set_option(mc_handle h, int option, int64_t value)
{
    switch (option) {
    case MC_OPT_GUARD_MODE:
        if (value < 0 || value > 3) return fail(MC_ERR_INVALID, "guard mode %lld", (long long)value);
        h->guard_mode = (int)value;
        return MC_OK;
    case MC_OPT_TIMEOUT_MS:
        if (value < 1) return fail(MC_ERR_INVALID, "timeout must be >= 1 ms");
        h->timeout_ms = value;
        return MC_OK;
    case MC_OPT_CTAS:
        if (value < 0) return fail(MC_ERR_INVALID, "CTAs < 0");
        h->ctas_override = (int)value;
        return MC_OK;
    case MC_OPT_SKIP_PUBLISH:
        h->skip_ticket = value;
        return MC_OK;
    case MC_OPT_USE_GRAPH:
        h->use_graph = value ? 1 : 0;
        return MC_OK;
    case MC_OPT_POLICY:
        if (value < 0 || value > 1) return fail(MC_ERR_INVALID, "policy %lld", (long long)value);
        h->policy = (int)value;
        return MC_OK;
    case MC_OPT_DA:
        h->da_on = value ? 1 : 0;
        drop_graphs(h);
        return sync_descriptors(h);
    case MC_OPT_PAIRS:
        if (value < -1 || value > 1) return fail(MC_ERR_INVALID, "pairs mode %lld", (long long)value);
        h->pairs_opt = (int)value;
        drop_graphs(h);
        return MC_OK;
    case MC_OPT_DEEP_WINDOWS:
        if (value < 0 || value > 1) return fail(MC_ERR_INVALID, "deep windows %lld", (long long)value);
        h->deep_opt = (int)value;
        drop_graphs(h);
        return MC_OK;
    case MC_OPT_DRIFT_EVERY:
        if (value < 0) return fail(MC_ERR_INVALID, "drift check period %lld", (long long)value);
        h->drift_every = value;
        return MC_OK;
    case MC_OPT_DA_SWEEPS:
        if (value < 1 || value > 64) return fail(MC_ERR_INVALID, "sweeps per launch %lld", (long long)value);
        for (auto &c : h->chains)
            if (c.dda && c.da_k != value)
                return fail(MC_ERR_INVALID, "a chain's cell list is sized for %d sweeps per launch: set the option "
                                            "before mc_set_surrogate / mc_set_overlap_prefilter", c.da_k);
        h->da_sweeps = (int)value;
        drop_graphs(h);
        return MC_OK;
    case MC_OPT_SHARED_GUARD:
        if (value < 0 || value > 1) return fail(MC_ERR_INVALID, "shared guard %lld", (long long)value);
        h->gb_opt = (int)value;
        drop_graphs(h);
        return MC_OK;
    case MC_OPT_HELPERS:
        if (value < 0 || value > 1) return fail(MC_ERR_INVALID, "helpers %lld", (long long)value);
        if (value == 1 && h->occ_h < 1) return fail(MC_ERR_INVALID, "the helper-warp kernel does not fit an SM");
        h->helpers_opt = (int)value;
        drop_graphs(h);
        return MC_OK;
    default:
        return fail(MC_ERR_INVALID, "unknown option %d", option);
    }
}

int mc_set_option(mc_handle h, int option, int64_t value)
{
    int rc = check(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    rc = set_option(h, option, value);
    write_ctl(h);
    return rc;
}

int mc_get_option(mc_handle h, int option, int64_t *value)
{
    int rc = check(h);
    if (rc) return rc;
    if (!value) return fail(MC_ERR_INVALID, "NULL output");
    switch (option) {
    case MC_OPT_GUARD_MODE: *value = h->guard_mode; return MC_OK;
    case MC_OPT_TIMEOUT_MS: *value = h->timeout_ms; return MC_OK;
    case MC_OPT_CTAS: *value = h->ctas_override > 0 ? h->ctas_override : grid_for(h); return MC_OK;
    case MC_OPT_SKIP_PUBLISH: *value = h->skip_ticket; return MC_OK;
    case MC_OPT_USE_GRAPH: *value = h->use_graph; return MC_OK;
    case MC_OPT_POLICY: *value = h->policy; return MC_OK;
    case MC_OPT_DA: *value = h->da_on; return MC_OK;
    case MC_OPT_PAIRS: *value = pairs_on(h) ? 1 : 0; return MC_OK;
    case MC_OPT_DEEP_WINDOWS: *value = h->deep_opt; return MC_OK;
    case MC_OPT_DRIFT_EVERY: *value = h->drift_every; return MC_OK;
    case MC_OPT_HELPERS: *value = helpers_on(h) ? 1 : 0; return MC_OK;
    case MC_OPT_DA_SWEEPS: *value = h->da_sweeps; return MC_OK;
    case MC_OPT_SHARED_GUARD: *value = (h->gb_opt && h->d_gb) ? 1 : 0; return MC_OK;
    default: return fail(MC_ERR_INVALID, "unknown option %d", option);
    }
}

// Autotuner: time trial launches of every candidate (ticket order x CTA count)
// on a saved copy of every chain's state, keep the fastest, restore the state.
int mc_autotune(mc_handle h, int64_t trial_sweeps, int64_t *best_policy, int64_t *best_ctas, int64_t *best_shape,
                double *best_ms)
{
    int rc = check(h);
    if (rc) return rc;
    if (trial_sweeps < 1) return fail(MC_ERR_INVALID, "trial_sweeps < 1");
    CK(cudaStreamSynchronize(h->stream));
    // save
    struct Saved {
        std::vector<float> pos;
        uint64_t sweeps;
        double ledger;
        mc_stats_t st;
    };
    std::vector<Saved> saved(h->chains.size());
    for (size_t i = 0; i < h->chains.size(); ++i) {
        saved[i].pos.resize((size_t)h->chains[i].N * 3);
        rc = mc_get_state(h, (int)i, saved[i].pos.data(), &saved[i].sweeps, &saved[i].ledger, &saved[i].st);
        if (rc) return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // one candidate: warm launch (schedule and graph built outside the timing), then trial_sweeps timed
    auto trial = [&](double &ms_out) -> int {
        int r = enqueue_sweeps(h, 1);
        if (!r) r = finish(h);
        if (r) return r;
        cudaEventRecord(e0, h->stream);
        r = enqueue_sweeps(h, trial_sweeps);
        cudaEventRecord(e1, h->stream);
        if (!r) r = finish(h);
        if (r) return r;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_out = ms;
        return MC_OK;
    };
    // shape: bit 0 pairs mode, bit 1 deep windows, bit 2 helper warps (pairs mode and helpers exclude each other)
    auto apply_shape = [&](int sh) -> int {
        int r = set_option(h, MC_OPT_PAIRS, (sh & 1) ? 1 : 0);
        if (!r) r = set_option(h, MC_OPT_DEEP_WINDOWS, (sh >> 1) & 1);
        if (!r) r = set_option(h, MC_OPT_HELPERS, (sh >> 2) & 1);
        write_ctl(h);
        return r;
    };
    const int old_pairs = h->pairs_opt, old_deep = h->deep_opt, old_help = h->helpers_opt;
    double best = 1e300;
    int bshape = -1;
    // 1. kernel shape at the default work order and CTA count
    for (int sh = 0; sh < 8 && rc == 0; ++sh) {
        if ((sh & 1) && (sh & 4)) continue;
        if ((sh & 1) && (h->max_clusters < 1 || any_da(h))) continue;
        if ((sh & 4) && h->occ_h < 1) continue;
        if (apply_shape(sh)) {  // not available here: skip the candidate
            g_err.clear();
            continue;
        }
        double ms = 0.0;
        rc = trial(ms);
        if (!rc && ms < best) {
            best = ms;
            bshape = sh;
        }
    }
    if (!rc && bshape >= 0) rc = apply_shape(bshape);
    if (rc || bshape < 0) {
        h->pairs_opt = old_pairs;
        h->deep_opt = old_deep;
        h->helpers_opt = old_help;
        drop_graphs(h);
        write_ctl(h);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc ? rc : fail(MC_ERR_INVALID, "no kernel shape could run");
    }
    // 2. work order x persistent CTA count with that shape
    const int full = std::max(1, grid_for(h));
    const int old_policy = h->policy, old_ctas = h->ctas_override;
    std::vector<int> ctas = {full, std::max(1, (3 * full) / 4), std::max(1, full / 2)};
    best = 1e300;
    int bp = old_policy, bc = old_ctas;
    for (int pol = 0; pol < 2 && rc == 0; ++pol)
        for (int nc : ctas) {
            h->policy = pol;
            h->ctas_override = nc;
            double ms = 0.0;
            rc = trial(ms);
            if (rc) break;
            if (ms < best) {
                best = ms;
                bp = pol;
                bc = nc == full ? 0 : nc;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->policy = bp;
    h->ctas_override = bc;
    if (rc) return rc;
    for (size_t i = 0; i < h->chains.size(); ++i) {
        rc = mc_set_state(h, (int)i, saved[i].pos.data(), saved[i].sweeps, saved[i].ledger, &saved[i].st);
        if (rc) return rc;
    }
    if (best_policy) *best_policy = bp;
    if (best_ctas) *best_ctas = bc == 0 ? full : bc;
    if (best_shape) *best_shape = bshape;
    if (best_ms) *best_ms = best;
    return MC_OK;
}


// ---------------------------------------------------------------------------
// Delayed acceptance with the learned surrogate (see include/mc.h).

static int set_surrogate_impl(mc_handle h, int chain, const uint16_t *w_bf16, int64_t n_w, double r_c, int W);

// Free the delayed-acceptance / prefilter arrays of a chain (the stream is idle).
static void release_da(Chain &c)
{
    cudaFree(c.dda); cudaFree(c.d_w); cudaFree(c.d_w2n); cudaFree(c.d_cell_start); cudaFree(c.d_cell_ions);
    cudaFree(c.d_slot_of); cudaFree(c.d_cnt); cudaFree(c.d_cellid); cudaFree(c.d_fill); cudaFree(c.d_cell_pos);
    c.dda = nullptr; c.d_w = nullptr; c.d_w2n = nullptr; c.d_cell_start = nullptr; c.d_cell_ions = nullptr;
    c.d_slot_of = nullptr; c.d_cnt = nullptr; c.d_cellid = nullptr; c.d_fill = nullptr; c.d_cell_pos = nullptr;
    c.da = false;
    c.pf = false;
    c.ncell = 0;
}

int mc_set_surrogate(mc_handle h, int chain, const uint16_t *w_bf16, int64_t n_w, double r_c, int W)
{
    Range nv("mc_set_surrogate");
    const int rc = set_surrogate_impl(h, chain, w_bf16, n_w, r_c, W);
    if (check(h) == MC_OK) write_ctl(h);  // the stream is idle here; pairs mode follows the surrogate state
    return rc;
}

static int set_surrogate_impl(mc_handle h, int chain, const uint16_t *w_bf16, int64_t n_w, double r_c, int W)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    Chain &c = h->chains[chain];
    if (!w_bf16) {
        if (c.pf) release_da(c);  // removing the surrogate never leaves a prefilter behind
        c.da = false;
        drop_graphs(h);
        return sync_descriptors(h);
    }
    if (n_w != mcg::DA_NP) return fail(MC_ERR_INVALID, "the surrogate has %d weights, got %lld", mcg::DA_NP, (long long)n_w);
    if (!(r_c > 0.0) || !(r_c <= 5.0 * c.sigma)) return fail(MC_ERR_INVALID, "r_c = %g outside (0, 5 sigma]", r_c);
    if (W < 2) return fail(MC_ERR_INVALID, "exclusion depth W = %d below 2", W);
    std::vector<float> wf(mcg::DA_NP);
    for (int k = 0; k < mcg::DA_NP; ++k) {
        const uint32_t u = (uint32_t)w_bf16[k] << 16;
        std::memcpy(&wf[k], &u, 4);
        if (!std::isfinite(wf[k])) return fail(MC_ERR_INVALID, "weight %d is not finite", k);
    }
    // near-field reach: r_c plus the largest trial displacement plus the largest move of a candidate since the
    // launch's start (one per sweep, MC_OPT_DA_SWEEPS sweeps); cells of edge >= reach / 2, so the cells within two
    // of an ion's start cell hold every ion within r_c of its old or trial position at any time of the launch
    const double D = (double)(float)(2.0 * c.h);
    const double reach = (r_c + (1.0 + h->da_sweeps) * std::sqrt(3.0) * 0.5 * D) * (1.0 + 0x1p-8) + 1e-6;
    const int G = std::max(1, std::min(64, (int)std::floor(2.0 * c.R / (0.5 * reach))));
    // (re)allocate
    release_da(c);
    c.ncell = G * G * G;
    const size_t N = (size_t)c.N;
    CK(cudaMalloc(&c.dda, sizeof(mcg::DADev)));
    CK(cudaMalloc(&c.d_w, sizeof(uint16_t) * mcg::DA_NP));
    CK(cudaMalloc(&c.d_w2n, sizeof(float) * mcg::DA_H));
    CK(cudaMalloc(&c.d_cell_start, sizeof(int) * ((size_t)c.ncell + 1)));
    CK(cudaMalloc(&c.d_cnt, sizeof(int) * (size_t)c.ncell));
    CK(cudaMalloc(&c.d_fill, sizeof(int) * (size_t)c.ncell));
    CK(cudaMalloc(&c.d_cell_ions, sizeof(int) * N));
    CK(cudaMalloc(&c.d_slot_of, sizeof(int) * N));
    CK(cudaMalloc(&c.d_cellid, sizeof(int) * N));
    CK(cudaMalloc(&c.d_cell_pos, sizeof(float4) * N));
    std::vector<float> w2n(mcg::DA_H);
    for (int o = 0; o < mcg::DA_H; ++o) {
        double sum = 0.0;
        for (int i = 0; i < mcg::DA_H; ++i) sum += std::fabs((double)wf[mcg::DA_OFF_W2 + o * mcg::DA_H + i]);
        w2n[o] = std::nextafter((float)sum, 3.0e38f);
    }
    CK(cudaMemcpy(c.d_w, w_bf16, sizeof(uint16_t) * mcg::DA_NP, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.d_w2n, w2n.data(), sizeof(float) * mcg::DA_H, cudaMemcpyHostToDevice));
    mcg::DADev d{};
    d.w = c.d_w;
    d.w2n = c.d_w2n;
    d.cell_start = c.d_cell_start;
    d.cell_ions = c.d_cell_ions;
    d.cell_pos = c.d_cell_pos;
    d.slot_of = c.d_slot_of;
    d.rc2 = r_c * r_c;
    d.tw = 0.5 * r_c;
    d.rs = r_c - d.tw;
    d.rs2 = d.rs * d.rs;
    d.rs2_lo = std::nextafter((float)(d.rs2 * (1.0 - 0x1p-19)), 0.0f);
    d.rs2_hi = std::nextafter((float)(d.rs2 * (1.0 + 0x1p-19)), 3.0e38f);
    d.rs2_f = (float)d.rs2;
    d.c32_f = (float)(32.0 / (d.rc2 - d.rs2));
    d.rs_f = (float)d.rs;
    d.itw_f = (float)(1.0 / d.tw);
    d.R = c.R;
    d.rc2_lo = std::nextafter((float)(d.rc2 * (1.0 - 0x1p-19)), 0.0f);
    d.rc2_hi = std::nextafter((float)(d.rc2 * (1.0 + 0x1p-19)), 3.0e38f);
    d.nf_scale = (float)((double)G / (2.0 * c.R));
    d.nf_R = (float)c.R;
    d.nf_edge = (float)(2.0 * c.R / (double)G);
    d.reach2 = (float)(reach * reach * (1.0 + 0x1p-10));
    d.Rr = (float)c.R;
    d.nf_G = G;
    d.W = W;
    d.mlp_zero = 1;
    for (int k = 0; k < mcg::DA_NP; ++k)
        if (w_bf16[k] & 0x7fffu) d.mlp_zero = 0;
    c.hda = d;
    CK(cudaMemcpy(c.dda, &d, sizeof d, cudaMemcpyHostToDevice));
    c.da = true;
    c.da_k = h->da_sweeps;
    drop_graphs(h);
    return sync_descriptors(h);
}

// The overlap prefilter (see include/mc.h): the delayed-acceptance machinery with stage 1 reduced to the overlap test
// against counted ions, over a bucket cell list of edge >= half of sigma + the largest trial + the largest move
// of a candidate.
int mc_set_overlap_prefilter(mc_handle h, int chain, int W)
{
    Range nv("mc_set_overlap_prefilter");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (W != 0 && W < 2) return fail(MC_ERR_INVALID, "exclusion depth W = %d: 0 (off) or at least 2", W);
    CK(cudaStreamSynchronize(h->stream));
    Chain &c = h->chains[chain];
    if (W == 0) {
        if (c.pf) release_da(c);
        drop_graphs(h);
        rc = sync_descriptors(h);
        if (rc == MC_OK && check(h) == MC_OK) write_ctl(h);
        return rc;
    }
    release_da(c);
    const double D = (double)(float)(2.0 * c.h);
    const double mv = std::sqrt(3.0) * 0.5 * D;  // largest move of one ion (one per sweep)
    const int K = h->da_sweeps;                   // sweeps per launch (one cell list per launch)
    const double reach = (c.sigma + (1.0 + K) * mv) * (1.0 + 0x1p-8) + 1e-6;
    // cells of edge >= reach / 2 (the 5^3 stencil covers the reach), at most 256 per axis and 8 per ion
    const int gmax = std::min(256, std::max(1, (int)std::cbrt(8.0 * (double)c.N)));
    const int G = std::max(1, std::min(gmax, (int)std::floor(2.0 * c.R / (0.5 * reach))));
    const double edge = 2.0 * c.R / (double)G;
    // slots per cell: m^3 sub-cubes of diagonal below sigma (with slack for the FP32 cell index) hold at most one
    // ion each of a non-overlapping configuration
    const int m = std::max(1, (int)std::ceil((edge * (1.0 + 0x1p-8) + 1e-4) * std::sqrt(3.0) / (c.sigma * (1.0 - 0x1p-16))));
    // five ions at least sigma apart do not fit a cube of edge below 0.894 sigma (sqrt(5)/2 is the largest least
    // distance of five points in a unit cube); an ion past a full cell is only left out of the list anyway
    const int cap = (edge * (1.0 + 0x1p-8) + 1e-4 < 0.894 * c.sigma) ? 4 : std::min(64, m * m * m);
    c.ncell = G * G * G;
    const size_t slots = (size_t)c.ncell * (size_t)cap, N = (size_t)c.N;
    CK(cudaMalloc(&c.dda, sizeof(mcg::DADev)));
    CK(cudaMalloc(&c.d_cnt, sizeof(int) * (size_t)c.ncell));
    CK(cudaMalloc(&c.d_cell_pos, sizeof(float4) * slots));
    CK(cudaMalloc(&c.d_slot_of, sizeof(int) * N));
    mcg::DADev d{};
    d.cell_pos = c.d_cell_pos;
    d.slot_of = c.d_slot_of;
    d.cell_cnt = c.d_cnt;
    d.R = c.R;
    d.nf_scale = (float)((double)G / (2.0 * c.R));
    d.nf_R = (float)c.R;
    d.nf_edge = (float)edge;
    d.reach2 = (float)(reach * reach * (1.0 + 0x1p-10));
    const double orr = (c.sigma + K * mv) * (1.0 + 0x1p-8) + 1e-6;
    d.ovl_reach2 = (float)(orr * orr * (1.0 + 0x1p-10));
    d.Rr = (float)c.R;
    d.nf_G = G;
    d.W = W;
    d.mlp_zero = 1;
    d.cap = cap;
    d.prefilter = 1;
    c.hda = d;
    CK(cudaMemcpy(c.dda, &d, sizeof d, cudaMemcpyHostToDevice));
    c.da = true;
    c.pf = true;
    c.da_k = K;
    drop_graphs(h);
    rc = sync_descriptors(h);
    if (rc == MC_OK && check(h) == MC_OK) write_ctl(h);
    return rc;
}

int mc_da_samples(mc_handle h, int chain, float *v_pairs, float *y, uint8_t *valid)
{
    Range nv("mc_da_samples");
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!v_pairs || !y || !valid) return fail(MC_ERR_INVALID, "NULL output");
    Chain &c = h->chains[chain];
    if (!c.dda || c.pf) return fail(MC_ERR_INVALID, "chain %d has no surrogate set (mc_set_surrogate)", chain);
    CK(cudaStreamSynchronize(h->stream));
    const size_t N = (size_t)c.N;
    float *dV = nullptr, *dY = nullptr;
    unsigned char *dv = nullptr;
    CK(cudaMalloc(&dV, sizeof(float) * 66 * N));
    CK(cudaMalloc(&dY, sizeof(float) * N));
    CK(cudaMalloc(&dv, N));
    cudaError_t e = mcg_host::da_prep_launch(h->d_chains + chain, c.N, c.dda, c.ncell, c.d_cnt, c.d_cellid,
                                             c.d_cell_start, c.d_fill, c.d_cell_ions, c.d_cell_pos, c.d_slot_of,
                                             h->stream);
    if (e == cudaSuccess) e = mcg_host::da_sample_launch(h->d_chains + chain, c.dda, c.B, h->sm_count, dV, dY, dv, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v_pairs, dV, sizeof(float) * 66 * N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, dY, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(valid, dv, N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dV);
    cudaFree(dY);
    cudaFree(dv);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "training samples: %s", cudaGetErrorString(e));
    return MC_OK;
}

namespace {

// Device buffers of one forward/backward pass over npairs sample pairs.
struct MlpPass {
    float *G = nullptr, *Z = nullptr, *D = nullptr, *part = nullptr, *grad = nullptr;
    double *lp = nullptr;
    int nblocks = 0;
    long long cap = 0;
    ~MlpPass()
    {
        cudaFree(G); cudaFree(Z); cudaFree(D); cudaFree(part); cudaFree(grad); cudaFree(lp);
    }
    cudaError_t alloc(long long npairs, int sms)
    {
        cap = npairs;
        nblocks = std::max(1, sms);
        cudaError_t e;
        if ((e = cudaMalloc(&G, sizeof(float) * 2 * npairs)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&Z, sizeof(float) * 2 * npairs * 2 * mcg::DA_H)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D, sizeof(float) * 2 * npairs * (2 * mcg::DA_H + 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&part, sizeof(float) * (size_t)nblocks * mcg::DA_NP)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&grad, sizeof(float) * mcg::DA_NP)) != cudaSuccess) return e;
        return cudaMalloc(&lp, sizeof(double) * (size_t)((npairs + 255) / 256));
    }
    // loss partials and the gradient of the mean pair loss over npairs pairs starting at V / Y
    cudaError_t run(const unsigned short *w, const float *V, const float *Y, long long npairs, float inv_n, cudaStream_t st)
    {
        cudaError_t e = mcg_host::mlp_forward_launch(w, V, 2 * npairs, G, Z, st);
        if (e == cudaSuccess) e = mcg_host::mlp_backward_launch(w, Z, G, Y, npairs, inv_n, D, lp, st);
        if (e == cudaSuccess) e = mcg_host::mlp_wgrad_launch(V, Z, D, 2 * npairs, nblocks, part, grad, st);
        return e;
    }
};

int device_sms()
{
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

int mc_mlp_forward(const uint16_t *w_bf16, const float *v, int64_t n, float *g)
{
    if (!w_bf16 || !v || !g || n < 0) return fail(MC_ERR_INVALID, "bad arguments");
    if (n == 0) return MC_OK;
    unsigned short *dw = nullptr;
    float *dv = nullptr, *dg = nullptr;
    cudaError_t e = cudaMalloc(&dw, sizeof(uint16_t) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMalloc(&dv, sizeof(float) * mcg::DA_NIN * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dg, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dw, w_bf16, sizeof(uint16_t) * mcg::DA_NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dv, v, sizeof(float) * mcg::DA_NIN * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mcg_host::mlp_forward_launch(dw, dv, n, dg, nullptr, 0);
    if (e == cudaSuccess) e = cudaMemcpy(g, dg, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dw);
    cudaFree(dv);
    cudaFree(dg);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "mc_mlp_forward: %s", cudaGetErrorString(e));
    return MC_OK;
}

int mc_mlp_loss_grad(const uint16_t *w_bf16, const float *v_pairs, const float *y, int64_t n, double *loss, float *grad)
{
    if (!w_bf16 || !v_pairs || !y || n < 1) return fail(MC_ERR_INVALID, "bad arguments");
    unsigned short *dw = nullptr;
    float *dv = nullptr, *dy = nullptr;
    MlpPass pass;
    std::vector<double> lp((size_t)((n + 255) / 256));
    cudaError_t e = cudaMalloc(&dw, sizeof(uint16_t) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMalloc(&dv, sizeof(float) * 66 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = pass.alloc(n, device_sms());
    if (e == cudaSuccess) e = cudaMemcpy(dw, w_bf16, sizeof(uint16_t) * mcg::DA_NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dv, v_pairs, sizeof(float) * 66 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = pass.run(dw, dv, dy, n, 1.0f / (float)n, 0);
    if (e == cudaSuccess && grad) e = cudaMemcpy(grad, pass.grad, sizeof(float) * mcg::DA_NP, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lp.data(), pass.lp, sizeof(double) * lp.size(), cudaMemcpyDeviceToHost);
    cudaFree(dw);
    cudaFree(dv);
    cudaFree(dy);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "mc_mlp_loss_grad: %s", cudaGetErrorString(e));
    if (loss) {
        double s = 0.0;
        for (double x : lp) s += x;
        *loss = s / (double)n;
    }
    return MC_OK;
}

int mc_mlp_train(const float *v_pairs, const float *y, int64_t n, const uint16_t *w_init, int epochs, int batch,
                 float lr, uint16_t *w_out, double *loss_per_epoch)
{
    Range nv("mc_mlp_train");
    if (!v_pairs || !y || !w_init || !w_out || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0f))
        return fail(MC_ERR_INVALID, "bad arguments");
    const long long nb = std::min<long long>(batch, n);
    float *dv = nullptr, *dy = nullptr, *p = nullptr, *m = nullptr, *v = nullptr;
    unsigned short *wbf = nullptr;
    MlpPass pass;
    std::vector<float> p0(mcg::DA_NP);
    for (int k = 0; k < mcg::DA_NP; ++k) {
        const uint32_t u = (uint32_t)w_init[k] << 16;
        std::memcpy(&p0[k], &u, 4);
    }
    std::vector<double> lp((size_t)((nb + 255) / 256));
    cudaError_t e = cudaMalloc(&dv, sizeof(float) * 66 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(float) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMalloc(&m, sizeof(float) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMalloc(&v, sizeof(float) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMalloc(&wbf, sizeof(uint16_t) * mcg::DA_NP);
    if (e == cudaSuccess) e = pass.alloc(nb, device_sms());
    if (e == cudaSuccess) e = cudaMemcpy(dv, v_pairs, sizeof(float) * 66 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p, p0.data(), sizeof(float) * mcg::DA_NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m, 0, sizeof(float) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMemset(v, 0, sizeof(float) * mcg::DA_NP);
    if (e == cudaSuccess) e = cudaMemcpy(wbf, w_init, sizeof(uint16_t) * mcg::DA_NP, cudaMemcpyHostToDevice);
    long long t = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        double sum = 0.0;
        for (long long s0 = 0; s0 < n && e == cudaSuccess; s0 += nb) {
            const long long np = std::min(nb, n - s0);
            e = pass.run(wbf, dv + 66 * s0, dy + s0, np, 1.0f / (float)np, 0);
            ++t;
            if (e == cudaSuccess)
                e = mcg_host::adam_launch(p, m, v, pass.grad, lr, b1, b2, 1e-8f, 1.0f - std::pow(b1, (float)t),
                                          1.0f - std::pow(b2, (float)t), wbf, 0);
            if (e == cudaSuccess) e = cudaMemcpy(lp.data(), pass.lp, sizeof(double) * (size_t)((np + 255) / 256), cudaMemcpyDeviceToHost);
            for (long long q = 0; q < (np + 255) / 256; ++q) sum += lp[(size_t)q];
        }
        if (loss_per_epoch) loss_per_epoch[ep] = sum / (double)n;
    }
    if (e == cudaSuccess) e = cudaMemcpy(w_out, wbf, sizeof(uint16_t) * mcg::DA_NP, cudaMemcpyDeviceToHost);
    cudaFree(dv);
    cudaFree(dy);
    cudaFree(p);
    cudaFree(m);
    cudaFree(v);
    cudaFree(wbf);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "mc_mlp_train: %s", cudaGetErrorString(e));
    return MC_OK;
}

void mc_destroy(mc_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    for (auto &s : h->scheds) cudaFree(s.second.first);
    for (auto &c : h->chains) free_chain(c);
    cudaFree(h->d_chains);
    cudaFree(h->d_ctl);
    cudaFree(h->d_gb);
    cudaFree(h->d_box);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

const char *mc_last_error(void)
{
    return g_err.c_str();
}

int mc_device_info(int *sm_count, int *sm_clock_khz, int *cc_major, int *cc_minor)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (sm_count) CK(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev));
    if (sm_clock_khz) CK(cudaDeviceGetAttribute(sm_clock_khz, cudaDevAttrClockRate, dev));
    if (cc_major) CK(cudaDeviceGetAttribute(cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    if (cc_minor) CK(cudaDeviceGetAttribute(cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    return MC_OK;
}

int mc_test_philox(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out_lib, uint32_t *out_curand)
{
    if (n < 1 || n > (1 << 24) || !ctr || !key || !out_lib || !out_curand) return fail(MC_ERR_INVALID, "bad arguments");
    uint4 *dc = nullptr, *dl = nullptr, *dr = nullptr;
    uint2 *dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, 16 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dl, 16 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dr, 16 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, 8 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mcg_host::philox_test_launch(dc, dk, (int)n, dl, dr, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out_lib, dl, 16 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_curand, dr, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dl);
    cudaFree(dr);
    cudaFree(dk);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "philox test: %s", cudaGetErrorString(e));
    return MC_OK;
}

int mc_unit_rates(double *rates)
{
    if (!rates) return fail(MC_ERR_INVALID, "NULL output");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(mcg_host::unit_rates(sms, rates));
    return MC_OK;
}

int mc_test_log(const double *u, int64_t n, double *out)
{
    if (n < 1 || n > (1 << 24) || !u || !out) return fail(MC_ERR_INVALID, "bad arguments");
    double *du = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&du, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 8 * n);
    if (e == cudaSuccess) e = cudaMemcpy(du, u, 8 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mcg_host::log_test_launch(du, (int)n, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 8 * n, cudaMemcpyDeviceToHost);
    cudaFree(du);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, "log test: %s", cudaGetErrorString(e));
    return MC_OK;
}

}  // extern "C"
