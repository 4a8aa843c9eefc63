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
 * Readings where the paper is silent:
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
    /* delayed-acceptance surrogate (NULL until mco_set_surrogate) */
    struct mco_da *da;
} mco_chain;

static void da_free(struct mco_da *d);

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
    da_free(c->da);
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

/* One trial move of ion i with move index m (Sec. 2 steps b-c; the selection, step a, is the caller's). */
static void one_move_m(mco_chain *c, uint64_t m, int64_t i)
{
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

/* One sequential trial move of ion i at sweep index s: move index s N + i. */
static void one_move(mco_chain *c, uint64_t s, int64_t i)
{
    one_move_m(c, s * (uint64_t)c->n + (uint64_t)i, i);
}

/* The ion selected by step m of the random updating scheme (Sec. 2, step a
 * "at random"): u = w1 2^32 + w0 from the draws of purpose 3 at move index
 * m, ion floor(u N / 2^64) (uniform up to N / 2^64).                          */
int64_t mco_random_index(const mco_chain *c, uint64_t m)
{
    uint32_t w[4];
    move_draws(c->seed, c->chain, m, 3u, w);
    const uint64_t u = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
    return (int64_t)(((unsigned __int128)u * (unsigned __int128)(uint64_t)c->n) >> 64);
}

/* n_cycles Monte Carlo cycles of the random updating scheme (Sec. 2): N steps
 * each, step t of cycle s moving the ion mco_random_index selects for move
 * index s N + t; every ion moves once per cycle on average.                  */
int mco_random_sweep(mco_chain *c, int64_t n_cycles)
{
    if (!c || n_cycles < 0) return MCO_ERR_INVALID;
    for (int64_t s = 0; s < n_cycles; ++s) {
        for (int64_t t = 0; t < c->n; ++t) {
            const uint64_t m = c->sweep * (uint64_t)c->n + (uint64_t)t;
            one_move_m(c, m, mco_random_index(c, m));
        }
        c->sweep++;
    }
    return MCO_OK;
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

/* ======================================================================== */
/* Delayed acceptance with a learned surrogate (a two-stage Metropolis test
 * in the sense of Christen & Fox, 2005).  The paper's method is the exact
 * sequential chain of Sec. 2; this variant keeps its stationary distribution
 * and skips the O(N) sum for moves that a cheap first stage already rejects.
 * Readings D1-D8:
 *
 *  D1 Surrogate energy of ion i at point p, given the others:
 *       Et(p) = l_B q_i [phi_near(p) + g(v(p))],
 *     phi_near(p) = sum q_j s(d) / d, d = |p - x_j|, over counted ions j with
 *     d^2 < r_c^2 (FP64 from FP32 coordinates, ascending j), s = 1 up to
 *     r_s = r_c / 2 and 1 - t^2 (3 - 2t), t = (d - r_s) / (r_c - r_s), beyond
 *     (a C1 taper: an ion crossing r_c changes phi_near continuously), and g
 *     the MLP below.  dEt = Et(x') - Et(x) is exactly antisymmetric.
 *  D2 Counted ions: all j != i except those tried in the W groups of 128
 *     ions preceding i's group in sweep order (cyclic over the sweep) and
 *     the earlier ions of i's own group.  The set depends only on the move
 *     index, so Et is a function of the current state for every move.
 *  D3 Features v(p): 32 shell net charges and the radial coordinate.  Shell k
 *     of p holds the counted ions j with r_s^2 <= d^2 < r_c^2 and
 *     floor(32 (d^2 - r_s^2) / (r_c^2 - r_s^2)) = k (FP64, clamped to 31):
 *     the taper region, where phi_near departs from the Coulomb sum.  A move
 *     changes these counts as ions cross shells, so g can learn the part of
 *     the energy change the taper leaves out.  v[k] = F[k] / 4, k < 32;
 *     v[32] = |p| / R (FP64).
 *  D4 g: 33-64-64-1 MLP, SiLU after both hidden layers, BF16 weights; the
 *     reference arithmetic is FP64 with sequential dot products (bias first),
 *     silu(z) = z / (1 + exp(-z)) with the exp below.
 *  D5 Stage 1: a trial that overlaps a counted ion is rejected; otherwise it
 *     passes iff u1 == 0 or dEt < -L(u1), u1 the acceptance draw of Philox
 *     purpose 0 (the plain chain's draw).
 *  D6 Stage 2 (survivors only): the exact sum of the plain chain (overlap
 *     with any ion rejects); accept iff u2 == 0 or fl(dE - dEt) < -L(u2), u2
 *     the fourth word of Philox purpose 1.  This is the delayed-acceptance
 *     ratio min(1, exp(-(dE - dEt))) for an antisymmetric dEt.
 *  D7 Outcomes: 0 accept, 1 stage-2 reject, 2 overlap, 3 wall, 4 stage-1
 *     reject.  The ledger adds the exact dE of accepted moves.
 *  D8 Parameter layout (6401 values): W1[64][33], b1[64], W2[64][64],
 *     b2[64], W3[64], b3.
 */
#define MCO_DA_S 128
#define MCO_DA_NIN 33
#define MCO_DA_H 64
#define MCO_DA_NP (MCO_DA_H * MCO_DA_NIN + MCO_DA_H + MCO_DA_H * MCO_DA_H + MCO_DA_H + MCO_DA_H + 1)
#define MCO_DA_REJECT1 4

struct mco_da {
    double w[MCO_DA_NP]; /* the BF16 weights, exactly, in FP64 */
    double rc, rc2, rs, tw, rs2; /* cutoff, its square, taper start and width, taper start squared */
    int W;
    uint64_t n_rej1, n_ovl1, n_ovl2, n_rej2;
    void *rec;
    int64_t rec_cap, rec_len;
};

typedef struct {
    uint64_t m;
    int32_t i;
    int32_t outcome; /* D7 */
    int32_t stage;   /* 1 if decided by stage 1 (or the wall), 2 if by the exact stage */
    int32_t pad;
    double dE;       /* exact dE (NaN unless stage 2 evaluated it) */
    double dEt;      /* surrogate dEt (NaN unless stage 1 evaluated it) */
    float a[3];
    float pad2;
} mco_da_record;

static void da_free(struct mco_da *d)
{
    free(d);
}

/* exp(x) in FP64 from +, -, *, / only (for the SiLU of reading D4, written
 * so that the reference and a device implementation of the same steps agree
 * bit for bit).  Method: x = k ln2 + r with k = round-half-even(x / ln2) and
 * r = (x - k ln2_head) - k ln2_tail (ln2_head has 32 significant bits, so
 * k ln2_head is exact); exp(r) = 1 + r(1 + r/2(1 + r/3(...(1 + r/20)))) by
 * nested Horner steps, |r| <= 0.35 so the truncation is below 2^-60; the
 * result is scaled by 2^k exactly.  exp(x) = 0 below -700 and +inf above
 * 709 by definition.                                                       */
double mco_exp(double x)
{
    if (x > 709.0) return INFINITY;
    if (x < -700.0) return 0.0;
    double kd = nearbyint(x / MCO_LN2_HEAD);
    double r = (x - kd * MCO_LN2_HEAD) - kd * MCO_LN2_TAIL;
    double p = 1.0;
    for (int k = 20; k >= 1; --k) p = 1.0 + (p * r) / (double)k;
    return ldexp(p, (int)kd);
}

static double silu64(double z)
{
    return z / (1.0 + mco_exp(-z));
}

/* Reading D4: g(v) with FP64 parameters w (layout D8). */
double mco_mlp_forward(const double *w, const double v[MCO_DA_NIN])
{
    const double *W1 = w, *b1 = W1 + MCO_DA_H * MCO_DA_NIN, *W2 = b1 + MCO_DA_H, *b2 = W2 + MCO_DA_H * MCO_DA_H;
    const double *W3 = b2 + MCO_DA_H, *b3 = W3 + MCO_DA_H;
    double h1[MCO_DA_H], h2[MCO_DA_H];
    for (int o = 0; o < MCO_DA_H; ++o) {
        double z = b1[o];
        for (int i = 0; i < MCO_DA_NIN; ++i) z = z + W1[o * MCO_DA_NIN + i] * v[i];
        h1[o] = silu64(z);
    }
    for (int o = 0; o < MCO_DA_H; ++o) {
        double z = b2[o];
        for (int i = 0; i < MCO_DA_H; ++i) z = z + W2[o * MCO_DA_H + i] * h1[i];
        h2[o] = silu64(z);
    }
    double g = b3[0];
    for (int i = 0; i < MCO_DA_H; ++i) g = g + W3[i] * h2[i];
    return g;
}

/* Adds scale * d g(v) / d w to grad (backpropagation through D4). */
static void mlp_grad_acc(const double *w, const double v[MCO_DA_NIN], double scale, double *grad)
{
    const double *W1 = w, *b1 = W1 + MCO_DA_H * MCO_DA_NIN, *W2 = b1 + MCO_DA_H, *b2 = W2 + MCO_DA_H * MCO_DA_H;
    const double *W3 = b2 + MCO_DA_H;
    double *gW1 = grad, *gb1 = gW1 + MCO_DA_H * MCO_DA_NIN, *gW2 = gb1 + MCO_DA_H, *gb2 = gW2 + MCO_DA_H * MCO_DA_H;
    double *gW3 = gb2 + MCO_DA_H, *gb3 = gW3 + MCO_DA_H;
    double z1[MCO_DA_H], h1[MCO_DA_H], z2[MCO_DA_H], h2[MCO_DA_H], d2[MCO_DA_H], d1[MCO_DA_H];
    for (int o = 0; o < MCO_DA_H; ++o) {
        double z = b1[o];
        for (int i = 0; i < MCO_DA_NIN; ++i) z = z + W1[o * MCO_DA_NIN + i] * v[i];
        z1[o] = z;
        h1[o] = silu64(z);
    }
    for (int o = 0; o < MCO_DA_H; ++o) {
        double z = b2[o];
        for (int i = 0; i < MCO_DA_H; ++i) z = z + W2[o * MCO_DA_H + i] * h1[i];
        z2[o] = z;
        h2[o] = silu64(z);
    }
    /* silu'(z) = s (1 + z (1 - s)), s = 1 / (1 + exp(-z)) */
    for (int o = 0; o < MCO_DA_H; ++o) {
        gW3[o] += scale * h2[o];
        double sg = 1.0 / (1.0 + mco_exp(-z2[o]));
        d2[o] = scale * W3[o] * (sg * (1.0 + z2[o] * (1.0 - sg)));
    }
    gb3[0] += scale;
    for (int i = 0; i < MCO_DA_H; ++i) d1[i] = 0.0;
    for (int o = 0; o < MCO_DA_H; ++o) {
        gb2[o] += d2[o];
        for (int i = 0; i < MCO_DA_H; ++i) {
            gW2[o * MCO_DA_H + i] += d2[o] * h1[i];
            d1[i] += d2[o] * W2[o * MCO_DA_H + i];
        }
    }
    for (int o = 0; o < MCO_DA_H; ++o) {
        double sg = 1.0 / (1.0 + mco_exp(-z1[o]));
        double dz = d1[o] * (sg * (1.0 + z1[o] * (1.0 - sg)));
        gb1[o] += dz;
        for (int i = 0; i < MCO_DA_NIN; ++i) gW1[o * MCO_DA_NIN + i] += dz * v[i];
    }
}

/* Training loss of the surrogate on n pairs (v0 = features at the old position, v1 at the trial, y = the
 * far part of the exact energy change in units of l_B q_i): mean of (g(v1) - g(v0) - y)^2, and its gradient
 * with respect to the FP64 parameters (grad may be NULL).                                                 */
double mco_mlp_loss_grad(const double *w, int64_t n, const double *v0, const double *v1, const double *y,
                         double *grad)
{
    if (grad)
        for (int k = 0; k < MCO_DA_NP; ++k) grad[k] = 0.0;
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        double r = (mco_mlp_forward(w, v1 + s * MCO_DA_NIN) - mco_mlp_forward(w, v0 + s * MCO_DA_NIN)) - y[s];
        loss += r * r;
        if (grad) {
            mlp_grad_acc(w, v1 + s * MCO_DA_NIN, 2.0 * r / (double)n, grad);
            mlp_grad_acc(w, v0 + s * MCO_DA_NIN, -2.0 * r / (double)n, grad);
        }
    }
    return loss / (double)n;
}

int mco_mlp_nparams(void)
{
    return MCO_DA_NP;
}

static double bf16_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Reading D2: is ion j counted for the move of ion i? */
static int da_counted(const mco_chain *c, int64_t i, int64_t j)
{
    if (j == i) return 0;
    int64_t B = (c->n + MCO_DA_S - 1) / MCO_DA_S;
    int64_t gi = i / MCO_DA_S, gj = j / MCO_DA_S;
    if (gj == gi) return j > i;
    int64_t back = ((gi - gj) % B + B) % B; /* groups from j's back to i's, 1 .. B-1 */
    int64_t w = c->da->W < B - 1 ? c->da->W : B - 1;
    return back > w;
}

/* Stage-1 quantities of ion i at point p (readings D1-D3): features v, the near-field potential and, when
 * is_trial, the overlap with a counted ion.                                                              */
static void da_point(const mco_chain *c, int64_t i, const float p[3], int is_trial, double v[MCO_DA_NIN], double *phi,
                     int *ovl)
{
    struct mco_da *d = c->da;
    double ph = 0.0;
    int o = 0;
    int F[32];
    for (int k = 0; k < 32; ++k) F[k] = 0;
    for (int64_t j = 0; j < c->n; ++j) {
        if (!da_counted(c, i, j)) continue;
        const float *y = c->x + 3 * j;
        double dx = (double)p[0] - (double)y[0];
        double dy = (double)p[1] - (double)y[1];
        double dz = (double)p[2] - (double)y[2];
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (is_trial && d2 < c->sig2) o = 1;
        if (d2 < d->rc2) {
            double dd = sqrt(d2);
            if (dd <= d->rs) {
                ph = ph + c->q[j] / dd;
            } else {
                double t = (dd - d->rs) / d->tw;
                double sw = 1.0 - (t * t) * (3.0 - 2.0 * t);
                ph = ph + c->q[j] * sw / dd;
            }
            if (d2 >= d->rs2) {
                int k = (int)floor(((d2 - d->rs2) / (d->rc2 - d->rs2)) * 32.0);
                F[k > 31 ? 31 : k] += (int)c->q[j];
            }
        }
    }
    for (int k = 0; k < 32; ++k) v[k] = (double)F[k] * 0.25;
    v[32] = sqrt(((double)p[0] * (double)p[0] + (double)p[1] * (double)p[1]) + (double)p[2] * (double)p[2]) / c->R;
    *phi = ph;
    if (ovl) *ovl = o;
}

/* Install the surrogate: n_w = 6401 BF16 weights (layout D8), near-field cutoff r_c, exclusion depth W. */
int mco_set_surrogate(mco_chain *c, const uint16_t *w_bf16, int64_t n_w, double r_c, int W)
{
    if (!c || !w_bf16 || n_w != MCO_DA_NP || !(r_c > 0.0) || W < 0) return MCO_ERR_INVALID;
    struct mco_da *d = c->da;
    if (!d) {
        d = (struct mco_da *)calloc(1, sizeof(struct mco_da));
        if (!d) return MCO_ERR_OOM;
        c->da = d;
    }
    for (int k = 0; k < MCO_DA_NP; ++k) d->w[k] = bf16_to_double(w_bf16[k]);
    d->rc = r_c;
    d->rc2 = r_c * r_c;
    d->tw = 0.5 * r_c;
    d->rs = r_c - d->tw;
    d->rs2 = d->rs * d->rs;
    d->W = W;
    return MCO_OK;
}

/* One delayed-acceptance move (readings D1-D7). */
static void one_move_da(mco_chain *c, uint64_t s, int64_t i)
{
    struct mco_da *d = c->da;
    uint64_t m = s * (uint64_t)c->n + (uint64_t)i;
    float a[3];
    uint32_t u1 = trial(c, m, i, a);
    float b[3] = {c->x[3 * i], c->x[3 * i + 1], c->x[3 * i + 2]};
    int outcome, stage = 1;
    double dE = NAN, dEt = NAN;
    double r2 = ((double)a[0] * (double)a[0] + (double)a[1] * (double)a[1]) + (double)a[2] * (double)a[2];
    if (r2 > c->Rc2) {
        outcome = MCO_REJECT_WALL;
    } else {
        double v1[MCO_DA_NIN], v0[MCO_DA_NIN], phi1, phi0;
        int ovl1 = 0;
        da_point(c, i, a, 1, v1, &phi1, &ovl1);
        if (ovl1) {
            outcome = MCO_REJECT_OVERLAP;
            d->n_ovl1++;
        } else {
            da_point(c, i, b, 0, v0, &phi0, NULL);
            dEt = (c->lB * c->q[i]) * ((phi1 + mco_mlp_forward(d->w, v1)) - (phi0 + mco_mlp_forward(d->w, v0)));
            if (!metropolis_accept(dEt, u1)) {
                outcome = MCO_DA_REJECT1;
                d->n_rej1++;
            } else {
                stage = 2;
                int ovl = 0;
                double total = canonical_sum(c, i, a, b, &ovl);
                if (ovl) {
                    outcome = MCO_REJECT_OVERLAP;
                    d->n_ovl2++;
                } else {
                    dE = (c->lB * c->q[i]) * total;
                    uint32_t w2[4];
                    move_draws(c->seed, c->chain, m, 1u, w2);
                    outcome = metropolis_accept(dE - dEt, w2[3] >> 8) ? MCO_ACCEPT : MCO_REJECT_METROPOLIS;
                    if (outcome == MCO_REJECT_METROPOLIS) d->n_rej2++;
                }
            }
        }
    }
    if (outcome == MCO_ACCEPT) {
        c->x[3 * i] = a[0];
        c->x[3 * i + 1] = a[1];
        c->x[3 * i + 2] = a[2];
        c->ledger = c->ledger + dE;
        c->n_accept++;
    } else if (outcome == MCO_REJECT_METROPOLIS || outcome == MCO_DA_REJECT1) {
        c->n_rej_metropolis++;
    } else if (outcome == MCO_REJECT_OVERLAP) {
        c->n_rej_overlap++;
    } else {
        c->n_rej_wall++;
    }
    if (d->rec && d->rec_len < d->rec_cap) {
        mco_da_record *r = (mco_da_record *)d->rec + d->rec_len++;
        r->m = m;
        r->i = (int32_t)i;
        r->outcome = outcome;
        r->stage = stage;
        r->pad = 0;
        r->dE = dE;
        r->dEt = dEt;
        r->a[0] = a[0];
        r->a[1] = a[1];
        r->a[2] = a[2];
        r->pad2 = 0.0f;
    }
}

/* n_sweeps delayed-acceptance cycles (same sequential order as mco_sweep). */
int mco_da_sweep(mco_chain *c, int64_t n_sweeps)
{
    if (!c || !c->da || n_sweeps < 0) return MCO_ERR_INVALID;
    for (int64_t s = 0; s < n_sweeps; ++s) {
        for (int64_t i = 0; i < c->n; ++i) one_move_da(c, c->sweep, i);
        c->sweep++;
    }
    return MCO_OK;
}

int mco_da_partial_sweep(mco_chain *c, int64_t n_moves)
{
    if (!c || !c->da || n_moves < 0 || n_moves > c->n) return MCO_ERR_INVALID;
    for (int64_t i = 0; i < n_moves; ++i) one_move_da(c, c->sweep, i);
    return MCO_OK;
}

/* DA counters: [stage-1 rejects, stage-1 overlaps, stage-2 overlaps, stage-2 rejects] */
int mco_da_stats(const mco_chain *c, uint64_t out[4])
{
    if (!c || !c->da || !out) return MCO_ERR_INVALID;
    out[0] = c->da->n_rej1;
    out[1] = c->da->n_ovl1;
    out[2] = c->da->n_ovl2;
    out[3] = c->da->n_rej2;
    return MCO_OK;
}

int mco_da_set_record(mco_chain *c, mco_da_record *buf, int64_t cap)
{
    if (!c || !c->da) return MCO_ERR_INVALID;
    c->da->rec = buf;
    c->da->rec_cap = buf ? cap : 0;
    c->da->rec_len = 0;
    return MCO_OK;
}

int64_t mco_da_record_len(const mco_chain *c)
{
    return (c && c->da) ? c->da->rec_len : 0;
}

/* Stage-1 quantities of a hypothetical move of ion i to a (no state change): features at the old and trial
 * positions, near-field potentials, trial overlap with a counted ion, and the surrogate dEt (NaN on overlap). */
int mco_da_probe(mco_chain *c, int64_t i, const float a[3], double v0[MCO_DA_NIN], double v1[MCO_DA_NIN], double phi[2],
                 int *ovl, double *dEt)
{
    if (!c || !c->da || i < 0 || i >= c->n) return MCO_ERR_INVALID;
    float b[3] = {c->x[3 * i], c->x[3 * i + 1], c->x[3 * i + 2]};
    da_point(c, i, b, 0, v0, &phi[0], NULL);
    da_point(c, i, a, 1, v1, &phi[1], ovl);
    struct mco_da *d = c->da;
    *dEt = *ovl ? NAN
                : (c->lB * c->q[i]) * ((phi[1] + mco_mlp_forward(d->w, v1)) - (phi[0] + mco_mlp_forward(d->w, v0)));
    return MCO_OK;
}
