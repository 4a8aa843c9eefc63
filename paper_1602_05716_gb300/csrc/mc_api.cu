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

namespace mcg_host {
size_t sweep_smem_bytes();
cudaError_t sweep_configure();
cudaError_t sweep_occupancy(int *blocks_per_sm);
cudaError_t sweep_launch(int grid, const mcg::ChainDev *chains, const mcg::Ticket *sched, int n_tickets, mcg::Ctl *ctl,
                         int n_chains, long long n_sweeps, cudaStream_t st);
cudaError_t energy_launch(const float4 *pos, int N, double lB, double *rows, double *out, cudaStream_t st);
cudaError_t gr_launch(const float4 *pos, int N, int n_bins, double dr, float rmax2_hi, int use_lim, double lim2,
                      unsigned long long *counts, cudaStream_t st);
cudaError_t philox_test_launch(const uint4 *ctr, const uint2 *key, int n, uint4 *out_lib, uint4 *out_curand,
                               cudaStream_t st);
cudaError_t log_test_launch(const double *u, int n, double *out, cudaStream_t st);
}  // namespace mcg_host

namespace {

thread_local std::string g_err;

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
    double *rows = nullptr;      // energy scratch (lazy)
    mcg::MoveRec *rec = nullptr;
    long long rec_cap = 0;
    mcg::TraceRec *trace = nullptr;
    long long trace_cap = 0;
    unsigned long long rec_sweep0 = 0;
    uint64_t sweeps = 0;         // host mirror of *sweep
    uint64_t sweep_base = 0;     // sweep count when the positions were last set from the host
    float4 *cur() const { return pos[sweeps & 1]; }
};

struct GraphKey {
    long long n;
    int grid;
    int policy;
    bool operator<(const GraphKey &o) const
    {
        return n != o.n ? n < o.n : (grid != o.grid ? grid < o.grid : policy < o.policy);
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
    return d;
}

int sync_descriptors(mc_system *h)
{
    h->h_chains.resize(h->chains.size());
    for (size_t i = 0; i < h->chains.size(); ++i) h->h_chains[i] = describe(h->chains[i]);
    CK(cudaMemcpy(h->d_chains, h->h_chains.data(), sizeof(mcg::ChainDev) * h->h_chains.size(), cudaMemcpyHostToDevice));
    return MC_OK;
}

int init_chain(mc_system *h, Chain &c, const mc_chain_desc &d)
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
    int rc = validate(d.pos_xyz, d.n, d.sigma, d.R);
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
    c.stats = (unsigned long long *)(c.slab + 64);  // NCOUNTERS counters
    rc = upload_positions(h, c, d.pos_xyz, h->stream);
    if (rc) return rc;
    CK(cudaMalloc(&c.rows, sizeof(double) * (size_t)c.N));
    CK(mcg_host::energy_launch(c.cur(), c.N, c.lB, c.rows, c.ledger, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

void free_chain(Chain &c)
{
    cudaFree(c.pos[0]);
    cudaFree(c.pos[1]);
    cudaFree(c.flags);
    cudaFree(c.bits);
    cudaFree(c.slab);
    cudaFree(c.rows);
    cudaFree(c.rec);
    cudaFree(c.trace);
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
        cudaMallocHost(&h->h_ctl, sizeof(mcg::Ctl)) != cudaSuccess)
        return bail(fail(MC_ERR_OOM, "allocation of launch state failed"));
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

int grid_for(mc_system *h)
{
    long long useful = 0;
    for (auto &c : h->chains) useful += c.B;
    long long g = (long long)h->sm_count * h->occ;
    if (h->ctas_override > 0) g = std::min<long long>(g, h->ctas_override);
    g = std::min(g, useful);
    return (int)std::max<long long>(1, g);
}

int enqueue_sweeps(mc_system *h, long long n)
{
    mcg::Ticket *sched = nullptr;
    int count = 0;
    int rc = schedule_for(h, n, &sched, &count);
    if (rc) return rc;
    const int grid = grid_for(h);
    const int nch = (int)h->chains.size();
    if (h->use_graph) {
        GraphKey key{n, grid, h->policy};
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(mcg::Ctl), cudaMemcpyHostToDevice, h->stream);
            cudaError_t e2 = mcg_host::sweep_launch(grid, h->d_chains, sched, count, h->d_ctl, nch, n, h->stream);
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
    } else {
        CK(cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(mcg::Ctl), cudaMemcpyHostToDevice, h->stream));
        CK(mcg_host::sweep_launch(grid, h->d_chains, sched, count, h->d_ctl, nch, n, h->stream));
    }
    for (auto &ch : h->chains) ch.sweeps += (uint64_t)n;
    return MC_OK;
}

// The pinned control block is copied to the device at the start of every
// launch (also inside captured graphs), so it is rewritten only while the
// stream is idle.
void write_ctl(mc_system *h)
{
    mcg::Ctl *c = h->h_ctl;
    std::memset(c, 0, sizeof(mcg::Ctl));
    c->guard_mode = h->guard_mode;
    c->timeout_ns = h->timeout_ms * 1000000ll;
    c->skip_ticket = h->skip_ticket;
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
    return create_common(descs, n_chains, out);
}

int mc_sweep_async(mc_handle h, int64_t n_sweeps)
{
    int rc = check(h);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(MC_ERR_INVALID, "n_sweeps < 0");
    if (n_sweeps == 0) return MC_OK;
    return enqueue_sweeps(h, n_sweeps);
}

int mc_synchronize(mc_handle h)
{
    int rc = check(h);
    if (rc) return rc;
    return finish(h);
}

int mc_sweep(mc_handle h, int64_t n_sweeps)
{
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
    int rc = check_chain(h, chain);
    if (rc) return rc;
    Chain &c = h->chains[chain];
    CK(cudaStreamSynchronize(h->stream));
    if (ledger) CK(cudaMemcpy(ledger, c.ledger, sizeof(double), cudaMemcpyDeviceToHost));
    if (recomputed) {
        CK(mcg_host::energy_launch(c.cur(), c.N, c.lB, c.rows, c.e_out, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaMemcpy(recomputed, c.e_out, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return MC_OK;
}

int mc_gr_histogram(mc_handle h, int chain, int n_bins, double r_max, double wall_margin, uint64_t *counts)
{
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

int mc_get_positions(mc_handle h, int chain, float *pos_xyz)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!pos_xyz) return fail(MC_ERR_INVALID, "NULL buffer");
    Chain &c = h->chains[chain];
    std::vector<float4> buf((size_t)c.N);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(buf.data(), c.cur(), sizeof(float4) * buf.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < c.N; ++i) {
        pos_xyz[3 * i] = buf[i].x;
        pos_xyz[3 * i + 1] = buf[i].y;
        pos_xyz[3 * i + 2] = buf[i].z;
    }
    return MC_OK;
}

int mc_set_positions(mc_handle h, int chain, const float *pos_xyz)
{
    int rc = check_chain(h, chain);
    if (rc) return rc;
    if (!pos_xyz) return fail(MC_ERR_INVALID, "NULL buffer");
    Chain &c = h->chains[chain];
    rc = validate(pos_xyz, c.N, c.sigma, c.R);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    rc = upload_positions(h, c, pos_xyz, h->stream);
    if (rc) return rc;
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
    default: return fail(MC_ERR_INVALID, "unknown option %d", option);
    }
}

// Autotuner: time trial launches of every candidate (ticket order x CTA count)
// on a saved copy of every chain's state, keep the fastest, restore the state.
int mc_autotune(mc_handle h, int64_t trial_sweeps, int64_t *best_policy, int64_t *best_ctas, double *best_ms)
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
    const int full = std::max(1, grid_for(h));
    const int old_policy = h->policy, old_ctas = h->ctas_override;
    std::vector<int> ctas = {full, std::max(1, (3 * full) / 4), std::max(1, full / 2)};
    double best = 1e300;
    int bp = old_policy, bc = old_ctas;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int pol = 0; pol < 2 && rc == 0; ++pol)
        for (int nc : ctas) {
            h->policy = pol;
            h->ctas_override = nc;
            rc = enqueue_sweeps(h, 1);  // warm: schedule and graph built outside the timing
            if (!rc) rc = finish(h);
            if (rc) break;
            cudaEventRecord(e0, h->stream);
            rc = enqueue_sweeps(h, trial_sweeps);
            cudaEventRecord(e1, h->stream);
            if (!rc) rc = finish(h);
            if (rc) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
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
    if (best_ms) *best_ms = best;
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
