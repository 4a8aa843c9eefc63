/*
 * mco.c -- plain, slow FP64 CPU oracle for the sequential Metropolis Monte
 * Carlo of primitive-model electrolytes (Liang, Xing & Li, "A GPU-based
 * Large-scale Monte Carlo Simulation Method for Systems with Long-range
 * Interactions", arXiv:1602.05716).
 *
 * TEST INFRASTRUCTURE.  The product library never links, includes or calls
 * anything in this directory; only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py use it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -shared
 * -fPIC.  -ffp-contract=off matters: every floating-point expression below is
 * a sequence of single IEEE-754 round-to-nearest operations in the order
 * written (aarch64 GCC would otherwise fuse multiply-adds).
 *
 * What is computed (paper section / equation / algorithm cited per function):
 *   - one Monte Carlo cycle ("sweep") = N sequential single-ion trial moves in
 *     ascending index order (Sec. 2, sequential updating scheme);
 *   - the energy change of move i uses the *current* positions of all other
 *     ions: already-moved ions j < i at their updated position, ions j > i at
 *     their position from the previous cycle (Sec. 2, the Delta E_ij table);
 *   - hard-core overlap indicator instead of an energy (Sec. 3.3);
 *   - acceptance when the uniform draw is below exp(-l_B * dE) (Algorithm 4,
 *     Eq. trial-outcome), l_B the Bjerrum length, energies in k_B T;
 *   - the hard spherical wall of Sec. 5.2.
 *
 * Readings where the paper is silent (each also listed in the design doc):
 *   R1 random numbers: Philox4x32-10 keyed by (seed, chain), counter = move
 *      index m = sweep*N + i, replacing the paper's host-side ran4 (Sec. 3.1);
 *   R2 u_k = (w_k >> 8) * 2^-24 (exact float in [0,1)); trial coordinate
 *      x'_k = fl32(x_k + fl32((u_k - 0.5f) * D)), D = fl32(2h) (Algorithm 1
 *      writes only the displacement; the new coordinate is old + displacement);
 *   R3 wall: reject if |x'|^2 > R_c^2, R_c = R - sigma/2 (centres confined so
 *      the whole sphere stays inside the hard wall of radius R);
 *   R4 overlap iff |x' - x_j|^2 < sigma^2 (contact allowed);
 *   R5 self energy 0 (uniform dielectric, no images);
 *   R6 accept iff u_acc == 0 or dE < -L(u_acc), strict, with L the FP64
 *      logarithm mco_log() below (the comparison u < exp(-dE) of Algorithm 4
 *      written in log form so that both implementations decide identically);
 *   R7 canonical summation: terms added sequentially within consecutive
 *      1024-index chunks of j, chunk sums then added sequentially.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MCO_OK 0
#define MCO_ERR_INVALID (-1)
#define MCO_ERR_OVERLAP_INIT (-2)
#define MCO_ERR_OOM (-5)

#define MCO_CHUNK 1024

/* outcome codes of a move record */
#define MCO_ACCEPT 0
#define MCO_REJECT_METROPOLIS 1
#define MCO_REJECT_OVERLAP 2
#define MCO_REJECT_WALL 3

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers, the key bumped by the published Weyl constants
 * between rounds.                                                          */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void mco_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* The four draws of move m of a chain (reading R1): counter (m_lo, m_hi,
 * purpose, seed_hi), key (seed_lo, chain).  purpose 0 = trial move and
 * acceptance, 1 = second stage of delayed acceptance.                     */
static void move_draws(uint64_t seed, uint32_t chain, uint64_t m, uint32_t purpose, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)(m >> 32), purpose, (uint32_t)(seed >> 32)};
    uint32_t key[2] = {(uint32_t)seed, chain};
    mco_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm in FP64 from +, -, *, / only (reading R6).  Method: the
 * argument reduction u = f * 2^e with f in [sqrt(1/2), sqrt(2)), then
 * ln f = 2 atanh(s), s = (f-1)/(f+1), by its Taylor series
 * 2 s (1 + s^2/3 + s^4/5 + ... + s^20/21) (Abramowitz & Stegun 4.1.27);
 * |s| <= 0.1716 so the first omitted term is below 2^-56 relative.  ln 2 is
 * split into a head with 32 significant bits (so e * head is exact) and a
 * tail.  Defined for u in (0, 1] (it is only ever called with u > 0).     */
#define MCO_LN2_HEAD 0.693147180601954460144042968750
#define MCO_LN2_TAIL (-4.2009150726810847291823431924e-11)
#define MCO_SQRT_HALF 0.70710678118654752440

double mco_log(double u)
{
    int e;
    double f = frexp(u, &e); /* u = f * 2^e, f in [0.5, 1) -- exact */
    if (f < MCO_SQRT_HALF) {
        f = f * 2.0; /* exact */
        e = e - 1;
    }
    double s = (f - 1.0) / (f + 1.0);
    double z = s * s;
    double p = 1.0 / 21.0;
    for (int k = 9; k >= 0; --k) {
        p = p * z + 1.0 / (double)(2 * k + 1);
    }
    double lnf = (2.0 * s) * p;
    double de = (double)e;
    return de * MCO_LN2_HEAD + (de * MCO_LN2_TAIL + lnf);
}

/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t m;      /* move index sweep*N + i */
    int32_t i;       /* ion moved */
    int32_t outcome; /* MCO_ACCEPT / ..._METROPOLIS / ..._OVERLAP / ..._WALL */
    double dE;       /* l_B q_i sum_j q_j (1/r' - 1/r) in k_B T; NaN if not evaluated */
    float a[3];      /* trial position */
    float pad;
    double scale;    /* l_B |q_i| sum_{j != i} |q_j| (1/r' + 1/r): the scale of the FP32 tolerance; NaN if not evaluated */
} mco_record;

typedef struct {
    int64_t n;
    float *x;   /* n*3 positions, FP32 as stored by the method (Sec. 3.1) */
    double *q;  /* valences */
    double sigma, sig2, lB, R, Rc, Rc2, h;
    float D;    /* fl32(2h): full edge of the trial cube (Algorithm 1's D) */
    uint64_t seed;
    uint32_t chain;
    uint64_t sweep; /* sweeps completed since creation */
    double ledger;  /* running sum of accepted dE since creation */
    double e0;      /* brute-force energy at creation (computed on first use) */
    int have_e0;
    uint64_t n_accept, n_rej_metropolis, n_rej_overlap, n_rej_wall;
    /* optional per-move record sink */
    mco_record *rec;
    int64_t rec_cap, rec_len;
    /* scratch for the chunked sums */
    double *chunk_sum;
    int *chunk_ovl;
    int64_t n_chunks;
} mco_chain;

static int nthreads_cfg = 1;

double mco_total_energy_of(const float *x, const double *q, int64_t n, double l_B);

void mco_set_threads(int n)
{
    nthreads_cfg = n < 1 ? 1 : n;
}

int mco_get_threads(void)
{
    return nthreads_cfg;
}

/* Pairwise overlap check of a configuration on a uniform grid (cell edge
 * >= sigma), plus the wall (readings R3, R4).  Returns 1 if valid.         */
static int config_valid(const float *x, int64_t n, double sig2, double sigma, double Rc2, double Rc)
{
    for (int64_t i = 0; i < n; ++i) {
        double a0 = x[3 * i], a1 = x[3 * i + 1], a2 = x[3 * i + 2];
        double r2 = (a0 * a0 + a1 * a1) + a2 * a2;
        if (!(r2 <= Rc2)) return 0;
    }
    double cell = sigma;
    int64_t m = (int64_t)floor(2.0 * Rc / cell) + 1;
    if (m > 512) {
        m = 512;
        cell = 2.0 * Rc / 511.0;
        if (cell < sigma) cell = sigma;
    }
    if (m < 1) m = 1;
    int64_t ncell = m * m * m;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!head || !next) {
        free(head);
        free(next);
        return -1;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    int ok = 1;
    for (int64_t i = 0; i < n && ok; ++i) {
        int64_t ci[3];
        for (int k = 0; k < 3; ++k) {
            int64_t v = (int64_t)floor(((double)x[3 * i + k] + Rc) / cell);
            if (v < 0) v = 0;
            if (v >= m) v = m - 1;
            ci[k] = v;
        }
        for (int64_t dx = -1; dx <= 1 && ok; ++dx)
            for (int64_t dy = -1; dy <= 1 && ok; ++dy)
                for (int64_t dz = -1; dz <= 1 && ok; ++dz) {
                    int64_t cx = ci[0] + dx, cy = ci[1] + dy, cz = ci[2] + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= m || cy >= m || cz >= m) continue;
                    for (int64_t j = head[(cx * m + cy) * m + cz]; j >= 0; j = next[j]) {
                        double d0 = (double)x[3 * i] - (double)x[3 * j];
                        double d1 = (double)x[3 * i + 1] - (double)x[3 * j + 1];
                        double d2 = (double)x[3 * i + 2] - (double)x[3 * j + 2];
                        double dd = (d0 * d0 + d1 * d1) + d2 * d2;
                        if (dd < sig2) ok = 0;
                    }
                }
        int64_t c = (ci[0] * m + ci[1]) * m + ci[2];
        next[i] = head[c];
        head[c] = i;
    }
    free(head);
    free(next);
    return ok;
}

int mco_create(const float *pos_xyz, const float *q, int64_t n, double sigma, double l_B,
               double R, double half_width, uint64_t seed, uint32_t chain_id, mco_chain **out)
{
    if (!out || !pos_xyz || !q || n < 1 || !(sigma > 0.0) || !(l_B >= 0.0) ||
        !(R > 0.5 * sigma) || !(half_width >= 0.0))
        return MCO_ERR_INVALID;
    mco_chain *c = (mco_chain *)calloc(1, sizeof(mco_chain));
    if (!c) return MCO_ERR_OOM;
    c->n = n;
    c->x = (float *)malloc(sizeof(float) * 3 * (size_t)n);
    c->q = (double *)malloc(sizeof(double) * (size_t)n);
    c->n_chunks = (n + MCO_CHUNK - 1) / MCO_CHUNK;
    c->chunk_sum = (double *)malloc(sizeof(double) * (size_t)c->n_chunks);
    c->chunk_ovl = (int *)malloc(sizeof(int) * (size_t)c->n_chunks);
    if (!c->x || !c->q || !c->chunk_sum || !c->chunk_ovl) {
        free(c->x); free(c->q); free(c->chunk_sum); free(c->chunk_ovl); free(c);
        return MCO_ERR_OOM;
    }
    memcpy(c->x, pos_xyz, sizeof(float) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) c->q[i] = (double)q[i];
    c->sigma = sigma;
    c->sig2 = sigma * sigma;
    c->lB = l_B;
    c->R = R;
    c->Rc = R - 0.5 * sigma;
    c->Rc2 = c->Rc * c->Rc;
    c->h = half_width;
    c->D = (float)(2.0 * half_width);
    c->seed = seed;
    c->chain = chain_id;
    int v = config_valid(c->x, n, c->sig2, sigma, c->Rc2, c->Rc);
    if (v != 1) {
        free(c->x); free(c->q); free(c->chunk_sum); free(c->chunk_ovl); free(c);
        return v < 0 ? MCO_ERR_OOM : MCO_ERR_OVERLAP_INIT;
    }
    if (n <= 65536) {
        c->e0 = mco_total_energy_of(c->x, c->q, n, l_B);
        c->have_e0 = 1;
    }
    *out = c;
    return MCO_OK;
}

void mco_destroy(mco_chain *c)
{
    if (!c) return;
    free(c->x);
    free(c->q);
    free(c->chunk_sum);
    free(c->chunk_ovl);
    free(c);
}

/* One chunk of the canonical sum (reading R7) for trial a / old position b of
 * ion i: sequential FP64 adds of t_j = q_j (1/|a - x_j| - 1/|b - x_j|) over
 * j in [j0, j1), j != i, with the positions as they stand (Sec. 2: updated
 * for j < i, previous cycle for j > i).  Sets *ovl if any |a - x_j| < sigma.
 * Distances are formed in FP64 from the FP32 coordinates (Sec. 3.3).       */
static double chunk_terms(const mco_chain *c, int64_t i, const float a[3], const float b[3],
                          int64_t j0, int64_t j1, int *ovl)
{
    double s = 0.0;
    int o = 0;
    for (int64_t j = j0; j < j1; ++j) {
        if (j == i) continue;
        const float *y = c->x + 3 * j;
        double dxn = (double)a[0] - (double)y[0];
        double dyn = (double)a[1] - (double)y[1];
        double dzn = (double)a[2] - (double)y[2];
        double d2n = (dxn * dxn + dyn * dyn) + dzn * dzn;
        if (d2n < c->sig2) o = 1;
        double dxo = (double)b[0] - (double)y[0];
        double dyo = (double)b[1] - (double)y[1];
        double dzo = (double)b[2] - (double)y[2];
        double d2o = (dxo * dxo + dyo * dyo) + dzo * dzo;
        double t = c->q[j] * (1.0 / sqrt(d2n) - 1.0 / sqrt(d2o));
        s = s + t;
    }
    *ovl = o;
    return s;
}

/* Canonical sum over all j != i: chunk sums (possibly computed by several
 * threads -- each chunk is still one sequential loop) added in chunk order. */
static double canonical_sum(mco_chain *c, int64_t i, const float a[3], const float b[3], int *ovl)
{
    int64_t nc = c->n_chunks;
#ifdef _OPENMP
    int nt = nthreads_cfg;
    if (nt > 1 && nc > 1) {
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t k = 0; k < nc; ++k) {
            int64_t j0 = k * MCO_CHUNK;
            int64_t j1 = j0 + MCO_CHUNK < c->n ? j0 + MCO_CHUNK : c->n;
            c->chunk_sum[k] = chunk_terms(c, i, a, b, j0, j1, &c->chunk_ovl[k]);
        }
    } else
#endif
    {
        for (int64_t k = 0; k < nc; ++k) {
            int64_t j0 = k * MCO_CHUNK;
            int64_t j1 = j0 + MCO_CHUNK < c->n ? j0 + MCO_CHUNK : c->n;
            c->chunk_sum[k] = chunk_terms(c, i, a, b, j0, j1, &c->chunk_ovl[k]);
        }
    }
    double total = 0.0;
    int o = 0;
    for (int64_t k = 0; k < nc; ++k) {
        total = total + c->chunk_sum[k];
        o |= c->chunk_ovl[k];
    }
    *ovl = o;
    return total;
}

/* Scale of the per-move dE tolerance, l_B |q_i| sum_{j != i} |q_j| (1/r' + 1/r),
 * over the same positions as chunk_terms (FP64, sequential).  Only filled in
 * records; the decision never reads it.                                     */
static double move_scale(const mco_chain *c, int64_t i, const float a[3], const float b[3])
{
    double s = 0.0;
    for (int64_t j = 0; j < c->n; ++j) {
        if (j == i) continue;
        const float *y = c->x + 3 * j;
        double dxn = (double)a[0] - (double)y[0], dyn = (double)a[1] - (double)y[1], dzn = (double)a[2] - (double)y[2];
        double dxo = (double)b[0] - (double)y[0], dyo = (double)b[1] - (double)y[1], dzo = (double)b[2] - (double)y[2];
        double rn = sqrt((dxn * dxn + dyn * dyn) + dzn * dzn), ro = sqrt((dxo * dxo + dyo * dyo) + dzo * dzo);
        s += fabs(c->q[j]) * (1.0 / rn + 1.0 / ro);
    }
    return c->lB * fabs(c->q[i]) * s;
}

/* Trial position of move m for ion i (Algorithm 1 with reading R2). Returns
 * the acceptance draw's integer (w3 >> 8).                                   */
static uint32_t trial(const mco_chain *c, uint64_t m, int64_t i, float a[3])
{
    uint32_t w[4];
    move_draws(c->seed, c->chain, m, 0u, w);
    for (int k = 0; k < 3; ++k) {
        float u = (float)(w[k] >> 8) * 0x1p-24f;
        float d = (u - 0.5f) * c->D;
        a[k] = c->x[3 * i + k] + d;
    }
    return w[3] >> 8;
}

/* The Metropolis test of Algorithm 4 / Eq. trial-outcome in log form (R6). */
static int metropolis_accept(double dE, uint32_t uacc)
{
    if (uacc == 0u) return 1;
    double u = (double)uacc * 0x1p-24;
    return dE < -mco_log(u);
}

/* One sequential trial move of ion i at sweep index s (Sec. 2 steps a-c). */
static void one_move(mco_chain *c, uint64_t s, int64_t i)
{
    uint64_t m = s * (uint64_t)c->n + (uint64_t)i;
    float a[3];
    uint32_t uacc = trial(c, m, i, a);
    float b[3] = {c->x[3 * i], c->x[3 * i + 1], c->x[3 * i + 2]};
    int outcome;
    double dE = NAN;
    double r2 = ((double)a[0] * (double)a[0] + (double)a[1] * (double)a[1]) + (double)a[2] * (double)a[2];
    if (r2 > c->Rc2) {
        outcome = MCO_REJECT_WALL;
    } else {
        int ovl = 0;
        double total = canonical_sum(c, i, a, b, &ovl);
        if (ovl) {
            outcome = MCO_REJECT_OVERLAP;
        } else {
            dE = (c->lB * c->q[i]) * total;
            outcome = metropolis_accept(dE, uacc) ? MCO_ACCEPT : MCO_REJECT_METROPOLIS;
        }
    }
    if (outcome == MCO_ACCEPT) {
        c->x[3 * i] = a[0];
        c->x[3 * i + 1] = a[1];
        c->x[3 * i + 2] = a[2];
        c->ledger = c->ledger + dE;
        c->n_accept++;
    } else if (outcome == MCO_REJECT_METROPOLIS) {
        c->n_rej_metropolis++;
    } else if (outcome == MCO_REJECT_OVERLAP) {
        c->n_rej_overlap++;
    } else {
        c->n_rej_wall++;
    }
    if (c->rec && c->rec_len < c->rec_cap) {
        mco_record *r = &c->rec[c->rec_len++];
        r->m = m;
        r->i = (int32_t)i;
        r->outcome = outcome;
        r->dE = dE;
        r->a[0] = a[0];
        r->a[1] = a[1];
        r->a[2] = a[2];
        r->pad = 0.0f;
        r->scale = isnan(dE) ? NAN : move_scale(c, i, a, b);
    }
}

/* n_sweeps Monte Carlo cycles: ions 0..N-1 tried once each, in ascending
 * order (Sec. 2, sequential updating scheme).                               */
int mco_sweep(mco_chain *c, int64_t n_sweeps)
{
    if (!c || n_sweeps < 0) return MCO_ERR_INVALID;
    for (int64_t s = 0; s < n_sweeps; ++s) {
        for (int64_t i = 0; i < c->n; ++i) one_move(c, c->sweep, i);
        c->sweep++;
    }
    return MCO_OK;
}

/* Only the first n_moves moves of the next sweep (prefix runs for large N). */
int mco_partial_sweep(mco_chain *c, int64_t n_moves)
{
    if (!c || n_moves < 0 || n_moves > c->n) return MCO_ERR_INVALID;
    for (int64_t i = 0; i < n_moves; ++i) one_move(c, c->sweep, i);
    return MCO_OK;
}

/* Brute-force total energy E = l_B sum_{i<j} q_i q_j / r_ij in FP64
 * (the Coulomb energy of the primitive model, Sec. 5; no cutoff, no images). */
double mco_total_energy_of(const float *x, const double *q, int64_t n, double l_B)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double row = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            double d0 = (double)x[3 * i] - (double)x[3 * j];
            double d1 = (double)x[3 * i + 1] - (double)x[3 * j + 1];
            double d2 = (double)x[3 * i + 2] - (double)x[3 * j + 2];
            double r = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
            row = row + q[j] / r;
        }
        e = e + q[i] * row;
    }
    return l_B * e;
}

/* ledger = E(initial configuration) + sum of accepted dE; recomputed = the
 * brute-force energy of the current configuration.                          */
int mco_energy(mco_chain *c, double *ledger, double *recomputed)
{
    if (!c) return MCO_ERR_INVALID;
    if (ledger) {
        if (!c->have_e0) return MCO_ERR_INVALID;
        *ledger = c->e0 + c->ledger;
    }
    if (recomputed) *recomputed = mco_total_energy_of(c->x, c->q, c->n, c->lB);
    return MCO_OK;
}

/* Pair-distance histogram behind g_{++}, g_{+-}, g_{--} (Sec. 5.2, Fig. PCF):
 * for every ion i whose centre satisfies |r_i|^2 <= (R_c - margin)^2 (all ions
 * when margin <= 0; Sec. 5.2 excludes ions near the wall) and every j != i,
 * bin = floor(sqrt(d2)/dr), dr = r_max/n_bins, counted when bin < n_bins.
 * Class 0 = both valences positive, 2 = both negative, 1 = mixed.  Counts are
 * ADDED to counts[3*n_bins].                                                 */
int mco_gr_histogram(mco_chain *c, int n_bins, double r_max, double wall_margin, uint64_t *counts)
{
    if (!c || n_bins < 1 || !(r_max > 0.0) || !counts) return MCO_ERR_INVALID;
    double dr = r_max / (double)n_bins;
    double lim = c->Rc - wall_margin;
    double lim2 = lim * lim;
    for (int64_t i = 0; i < c->n; ++i) {
        const float *a = c->x + 3 * i;
        if (wall_margin > 0.0) {
            if (lim < 0.0) break;
            double r2 = ((double)a[0] * (double)a[0] + (double)a[1] * (double)a[1]) + (double)a[2] * (double)a[2];
            if (r2 > lim2) continue;
        }
        for (int64_t j = 0; j < c->n; ++j) {
            if (j == i) continue;
            const float *y = c->x + 3 * j;
            double d0 = (double)a[0] - (double)y[0];
            double d1 = (double)a[1] - (double)y[1];
            double d2 = (double)a[2] - (double)y[2];
            double r = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
            double fb = floor(r / dr);
            if (fb >= (double)n_bins) continue;
            int cls = (c->q[i] > 0.0 && c->q[j] > 0.0) ? 0 : ((c->q[i] < 0.0 && c->q[j] < 0.0) ? 2 : 1);
            counts[(size_t)cls * (size_t)n_bins + (size_t)fb] += 1u;
        }
    }
    return MCO_OK;
}

int mco_get_positions(const mco_chain *c, float *pos_xyz)
{
    if (!c || !pos_xyz) return MCO_ERR_INVALID;
    memcpy(pos_xyz, c->x, sizeof(float) * 3 * (size_t)c->n);
    return MCO_OK;
}

/* Replace positions (checkpoint restore); validated like mco_create. */
int mco_set_positions(mco_chain *c, const float *pos_xyz)
{
    if (!c || !pos_xyz) return MCO_ERR_INVALID;
    if (config_valid(pos_xyz, c->n, c->sig2, c->sigma, c->Rc2, c->Rc) != 1) return MCO_ERR_OVERLAP_INIT;
    memcpy(c->x, pos_xyz, sizeof(float) * 3 * (size_t)c->n);
    return MCO_OK;
}

/* counters: [sweep, accepts, rej_metropolis, rej_overlap, rej_wall] */
int mco_stats(const mco_chain *c, uint64_t out[5])
{
    if (!c || !out) return MCO_ERR_INVALID;
    out[0] = c->sweep;
    out[1] = c->n_accept;
    out[2] = c->n_rej_metropolis;
    out[3] = c->n_rej_overlap;
    out[4] = c->n_rej_wall;
    return MCO_OK;
}

/* Set sweep counter and ledger (checkpoint restore). */
/* Set the sweep counter and the ledger (checkpoint restore): afterwards
 * mco_energy reports `ledger` as the running energy.                        */
int mco_set_counters(mco_chain *c, uint64_t sweep, double ledger)
{
    if (!c) return MCO_ERR_INVALID;
    c->sweep = sweep;
    c->e0 = ledger;
    c->have_e0 = 1;
    c->ledger = 0.0;
    return MCO_OK;
}

/* Per-move records go to buf (capacity cap) until full; NULL disables. */
int mco_set_record(mco_chain *c, mco_record *buf, int64_t cap)
{
    if (!c) return MCO_ERR_INVALID;
    c->rec = buf;
    c->rec_cap = buf ? cap : 0;
    c->rec_len = 0;
    return MCO_OK;
}

int64_t mco_record_len(const mco_chain *c)
{
    return c ? c->rec_len : 0;
}

/* The canonical dE of a hypothetical move of ion i to a (no state change);
 * *ovl gets the overlap indicator.  Used by the pins and the error reports. */
double mco_delta_e(mco_chain *c, int64_t i, const float a[3], int *ovl)
{
    float b[3] = {c->x[3 * i], c->x[3 * i + 1], c->x[3 * i + 2]};
    double total = canonical_sum(c, i, a, b, ovl);
    return (c->lB * c->q[i]) * total;
}

/* The random draws of move m (exposed for the generator pins). */
void mco_move_draws(uint64_t seed, uint32_t chain, uint64_t m, uint32_t purpose, uint32_t w[4])
{
    move_draws(seed, chain, m, purpose, w);
}
