/*
 * mcx_oracle.c -- plain, slow, obviously-correct CPU FP64 oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Built with  gcc -O2 -ffp-contract=off  so that every floating-point
 * operation is the IEEE binary64 operation written in the source (no fused
 * multiply-add contraction, no reassociation).
 *
 * What it computes (paper: arXiv 2402.09222, Sec. 5.1, the description of the
 * tunable parameters of OpenMC's event-based mode):
 *   - the macroscopic cross-section lookup, "the most expensive kernel":
 *     for every species of a material, find the energy-grid interval that
 *     holds E, interpolate each reaction channel linearly and sum the
 *     density-weighted results.  The hash grid of the paper only narrows the
 *     search window, so the oracle is the plain definition: a full binary
 *     search over each species' grid;
 *   - the adjoint of that lookup (it is linear in densities and tables);
 *   - event-by-event fixed-source neutron transport (flight, surface
 *     crossing, collision, track-length tallies), history by history.  The
 *     particles-in-flight count, queueing mode and sorting threshold of the
 *     paper do not change any history, so the oracle has none of them;
 *   - likelihood-ratio derivative tallies w.r.t. material density scales;
 *   - the k-eigenvalue power iteration of the paper's reactor benchmark
 *     (Sec. 5.1: Hoogenboom-Martin, a criticality problem): generations of
 *     histories started from the previous generation's fission sites.
 * The paper gives no physics; the readings taken where it is silent are
 * stated beside each function.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written from that paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11, Sec. 4.2: the Philox S-box with W=32,  */
/* N=4, multipliers M0, M1 and Weyl key increments).                          */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Two 32-bit words -> a double in the open interval (0,1):
 * u = (k + 1/2) 2^-52 with k = the top 26 bits of a, then the top 26 bits of b.
 * k < 2^52, so k + 1/2 and the scaling are exact. */
static double orc_u01(uint32_t a, uint32_t b)
{
    uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return ((double)k + 0.5) * 0x1.0p-52;
}

typedef struct {
    uint32_t key[2];
    uint32_t hist_lo, hist_hi;
    uint32_t n; /* per-history draw index */
} orc_rng;

static void orc_rng_init(orc_rng* r, uint64_t seed, uint32_t problem_id, uint64_t hist)
{
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32) ^ problem_id;
    r->hist_lo = (uint32_t)hist;
    r->hist_hi = (uint32_t)(hist >> 32);
    r->n = 0;
}

/* Uniform number n of a history: block n/2 of the Philox stream keyed by
 * (seed, problem), counter (n/2, hist_lo, hist_hi, 0); even n takes words
 * 0,1 and odd n words 2,3. */
static double orc_draw(orc_rng* r)
{
    uint32_t ctr[4] = {r->n >> 1, r->hist_lo, r->hist_hi, 0u}, w[4];
    orc_philox4x32_10(ctr, r->key, w);
    double u = (r->n & 1u) ? orc_u01(w[2], w[3]) : orc_u01(w[0], w[1]);
    r->n += 1u;
    return u;
}

/* Exported for tests: `count` consecutive uniforms of one history. */
void orc_uniforms(uint64_t seed, uint32_t problem_id, uint64_t hist, uint32_t first,
                  int64_t count, double* out)
{
    orc_rng r;
    orc_rng_init(&r, seed, problem_id, hist);
    r.n = first;
    for (int64_t i = 0; i < count; ++i) out[i] = orc_draw(&r);
}

/* ------------------------------------------------------------------------ */
/* Grid search and interpolation (Sec. 5.1, hash-grid paragraph: a search of  */
/* each species' energy grid, then interpolation).                            */
/* ------------------------------------------------------------------------ */

/* k = the largest k in [0, n-2] with g[k] <= E; k = 0 when E < g[0] (or E is
 * NaN), k = n-2 when E >= g[n-1].  E == g[k] gives k.  Requires n >= 2 and a
 * strictly increasing grid. */
int64_t orc_grid_index(const double* g, int64_t n, double E)
{
    if (!(E >= g[0])) return 0;
    if (E >= g[n - 1]) return n - 2;
    int64_t lo = 0, hi = n - 1; /* g[lo] <= E < g[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g[mid] <= E) lo = mid;
        else hi = mid;
    }
    return lo;
}

/* Interpolation fraction on [g[k], g[k+1]], clamped to [0, 1]. */
static double orc_fraction(const double* g, int64_t k, double E)
{
    double f = (E - g[k]) / (g[k + 1] - g[k]);
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return f;
}

/* Macroscopic lookup: out[l][r] = sum_i N_i * sigma_{r,i}(E_l) over the
 * species i of material mat[l], in stored order, starting from +0.0, with
 * sigma = s[k] + f * (s[k+1] - s[k]).  Returns the number of lookups with an
 * out-of-range material id (their outputs are set to NaN). */
int64_t orc_xs_lookup(int32_t n_species, const int64_t* grid_offsets, const double* energies,
                      const double* sigma, int32_t n_ch, int32_t n_materials,
                      const int32_t* mat_offsets, const int32_t* mat_species,
                      const double* mat_dens, int64_t n, const double* E, const int32_t* mat,
                      double* out, int n_threads)
{
    int64_t bad = 0;
    (void)n_species;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static) reduction(+ : bad)
#endif
    for (int64_t l = 0; l < n; ++l) {
        double* o = out + l * n_ch;
        int32_t m = mat[l];
        if (m < 0 || m >= n_materials) {
            for (int r = 0; r < n_ch; ++r) o[r] = NAN;
            bad += 1;
            continue;
        }
        for (int r = 0; r < n_ch; ++r) o[r] = 0.0;
        for (int32_t i = mat_offsets[m]; i < mat_offsets[m + 1]; ++i) {
            int32_t s = mat_species[i];
            const double* g = energies + grid_offsets[s];
            int64_t np = grid_offsets[s + 1] - grid_offsets[s];
            const double* tab = sigma + grid_offsets[s] * n_ch;
            int64_t k = orc_grid_index(g, np, E[l]);
            double f = orc_fraction(g, k, E[l]);
            for (int r = 0; r < n_ch; ++r) {
                double s0 = tab[k * n_ch + r], s1 = tab[(k + 1) * n_ch + r];
                double sg = s0 + f * (s1 - s0);
                o[r] = o[r] + mat_dens[i] * sg;
            }
        }
    }
    return bad;
}

/* Per-(lookup, species) grid indices, for index parity tests:
 * kout[l * max_species + i] = k of the i-th species of material mat[l]
 * (entries past the material's species count are set to -1). */
void orc_xs_indices(const int64_t* grid_offsets, const double* energies,
                    const int32_t* mat_offsets, const int32_t* mat_species, int64_t n,
                    const double* E, const int32_t* mat, int32_t max_species, int32_t* kout)
{
    for (int64_t l = 0; l < n; ++l) {
        int32_t m = mat[l];
        int32_t cnt = mat_offsets[m + 1] - mat_offsets[m];
        for (int32_t i = 0; i < max_species; ++i) {
            if (i >= cnt) {
                kout[l * max_species + i] = -1;
                continue;
            }
            int32_t s = mat_species[mat_offsets[m] + i];
            kout[l * max_species + i] = (int32_t)orc_grid_index(
                energies + grid_offsets[s], grid_offsets[s + 1] - grid_offsets[s], E[l]);
        }
    }
}

/* Adjoint of orc_xs_lookup for a cotangent grad_out[l][r]:
 *   grad_dens[i]              += sum_r grad_out[l][r] * sigma_{r,i}(E_l)
 *   grad_sigma[p_k][r]        += N_i * (1 - f) * grad_out[l][r]
 *   grad_sigma[p_{k+1}][r]    += N_i * f * grad_out[l][r]
 * (the derivatives of sigma = (1-f) s[k] + f s[k+1]).  Accumulates into the
 * caller's (zeroed) arrays.  Sequential: lookups in order. */
void orc_xs_lookup_backward(const int64_t* grid_offsets, const double* energies,
                            const double* sigma, int32_t n_ch, const int32_t* mat_offsets,
                            const int32_t* mat_species, const double* mat_dens, int64_t n,
                            const double* E, const int32_t* mat, const double* grad_out,
                            double* grad_dens, double* grad_sigma)
{
    for (int64_t l = 0; l < n; ++l) {
        int32_t m = mat[l];
        const double* go = grad_out + l * n_ch;
        for (int32_t i = mat_offsets[m]; i < mat_offsets[m + 1]; ++i) {
            int32_t s = mat_species[i];
            const double* g = energies + grid_offsets[s];
            int64_t np = grid_offsets[s + 1] - grid_offsets[s];
            int64_t base = grid_offsets[s];
            int64_t k = orc_grid_index(g, np, E[l]);
            double f = orc_fraction(g, k, E[l]);
            for (int r = 0; r < n_ch; ++r) {
                double s0 = sigma[(base + k) * n_ch + r], s1 = sigma[(base + k + 1) * n_ch + r];
                double sg = s0 + f * (s1 - s0);
                grad_dens[i] += go[r] * sg;
                grad_sigma[(base + k) * n_ch + r] += mat_dens[i] * (1.0 - f) * go[r];
                grad_sigma[(base + k + 1) * n_ch + r] += mat_dens[i] * f * go[r];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Transport                                                                  */
/* ------------------------------------------------------------------------ */
enum { ORC_GEOM_INFINITE = 0, ORC_GEOM_LATTICE = 1, ORC_GEOM_SLAB = 2 };
enum { ORC_OUT_ABSORBED = 0, ORC_OUT_LEAK_XHI = 1, ORC_OUT_LEAK_OTHER = 2, ORC_OUT_CUTOFF = 3,
       ORC_OUT_COLLISIONS = 4, ORC_N_OUT = 5 };
enum { ORC_S_NONE = 0, ORC_S_ZTOP, ORC_S_ZBOT, ORC_S_CYL, ORC_S_XLO, ORC_S_XHI, ORC_S_YLO,
       ORC_S_YHI };
#define ORC_MAX_DMAT 16
#define ORC_MAX_EVENTS_PER_HISTORY 100000000LL
#define ORC_MAX_AZIMUTH_TRIES 64

typedef struct {
    int32_t geometry;
    int32_t lattice_n;
    double pitch, radius, height, slab_length;
    int32_t n_regions;
    const int32_t* region_material;
    double E0, E_cut;
    int32_t n_ebins;
    const double* ebin_edges; /* n_ebins + 1 */
    int32_t n_batches;
    uint32_t problem_id;
    int64_t n_histories_total;
    /* library */
    int32_t n_species;
    const int64_t* grid_offsets;
    const double* energies;
    const double* sigma; /* [points][n_ch] */
    int32_t n_ch;
    int32_t ch_scatter, ch_absorb;
    const double* awr;
    int32_t n_materials;
    const int32_t* mat_offsets;
    const int32_t* mat_species;
    const double* mat_dens;
    int32_t derivatives;
    int32_t ch_nu_fission; /* channel of nu-fission, or -1 (eigenvalue runs only) */
} orc_problem;

typedef struct {
    double* flux;     /* [B][nb] */
    double* absorb;   /* [B][nb] */
    double* outcome;  /* [B][5] */
    double* dflux;    /* [B][nb][M] (derivatives only) */
    double* dabsorb;  /* [B][nb][M] */
    double* doutcome; /* [B][5][M] */
    uint32_t* ncoll;  /* [n_histories] of this call, or NULL */
} orc_tallies;

static int32_t orc_n_bins(const orc_problem* p)
{
    if (p->geometry == ORC_GEOM_INFINITE) return p->n_ebins;
    return p->n_regions;
}

/* Transport macroscopic lookup at energy E in material m: the sequential sums
 * Sigma_t = sum_i N_i (sigma_s,i + sigma_a,i) and Sigma_a = sum_i N_i sigma_a,i,
 * and, when sig_nf is given, nu Sigma_f = sum_i N_i nu sigma_f,i. */
static void orc_macro(const orc_problem* p, int32_t m, double E, double* sig_t, double* sig_a,
                      double* sig_nf)
{
    double st = 0.0, sa = 0.0, nf = 0.0;
    for (int32_t i = p->mat_offsets[m]; i < p->mat_offsets[m + 1]; ++i) {
        int32_t s = p->mat_species[i];
        const double* g = p->energies + p->grid_offsets[s];
        int64_t np = p->grid_offsets[s + 1] - p->grid_offsets[s];
        const double* tab = p->sigma + p->grid_offsets[s] * p->n_ch;
        int64_t k = orc_grid_index(g, np, E);
        double f = orc_fraction(g, k, E);
        double s0 = tab[k * p->n_ch + p->ch_scatter], s1 = tab[(k + 1) * p->n_ch + p->ch_scatter];
        double a0 = tab[k * p->n_ch + p->ch_absorb], a1 = tab[(k + 1) * p->n_ch + p->ch_absorb];
        double ss = s0 + f * (s1 - s0);
        double sa_i = a0 + f * (a1 - a0);
        st = st + p->mat_dens[i] * (ss + sa_i);
        sa = sa + p->mat_dens[i] * sa_i;
        if (sig_nf) {
            double n0 = tab[k * p->n_ch + p->ch_nu_fission], n1 = tab[(k + 1) * p->n_ch + p->ch_nu_fission];
            nf = nf + p->mat_dens[i] * (n0 + f * (n1 - n0));
        }
    }
    *sig_t = st;
    *sig_a = sa;
    if (sig_nf) *sig_nf = nf;
}

/* Azimuth (cos phi, sin phi) by rejection from pairs (a, b) = (2u-1, 2u-1)
 * with 0 < a^2 + b^2 <= 1. */
static void orc_azimuth(orc_rng* r, double* c, double* s)
{
    for (int t = 0; t < ORC_MAX_AZIMUTH_TRIES; ++t) {
        double a = 2.0 * orc_draw(r) - 1.0;
        double b = 2.0 * orc_draw(r) - 1.0;
        double rho = a * a + b * b;
        if (rho > 0.0 && rho <= 1.0) {
            *c = (a * a - b * b) / rho;
            *s = 2.0 * a * b / rho;
            return;
        }
    }
    *c = 1.0;
    *s = 0.0;
}

typedef struct {
    double x, y, z, u, v, w, E;
    int32_t ci, cj, inpin, region, material;
    int alive;
    int need_xs;
    double sig_t, sig_a, sig_nf;
    double W[ORC_MAX_DMAT];
    uint32_t ncoll;
} orc_particle;

/* A fission site: where a collision produced fission neutrons, with the
 * lattice cell and the inside-pin flag there (the region follows). */
typedef struct {
    double x, y, z;
    int32_t ci, cj, inpin;
} orc_site;

/* Eigenvalue context of one history. */
typedef struct {
    double k_norm;        /* a collision banks floor(nuSigma_f / Sigma_t / k_norm + xi) sites */
    double T;             /* temperature of the fission spectrum (eV) */
    const orc_site* src;  /* this history's source site, or NULL (the fixed source) */
    orc_site* sites;      /* sites this history banked (grown with realloc) */
    int64_t n_sites, cap_sites;
    double k_col, k_tl;   /* this history's collision and track-length k scores */
    int failed;           /* out of memory */
} orc_eigen;

static void orc_set_region(const orc_problem* p, orc_particle* q)
{
    if (p->geometry == ORC_GEOM_LATTICE) {
        int32_t n = p->lattice_n;
        q->region = q->inpin ? q->ci * n + q->cj : n * n;
    } else {
        q->region = 0;
    }
    q->material = p->region_material[q->region];
}

/* Source (BASELINE lattice workload: a pin centre chosen uniformly at
 * mid-height, isotropic, E0).  Infinite medium: origin, isotropic.  Slab:
 * pencil beam along +x at x = 0. */
static void orc_source(const orc_problem* p, orc_rng* r, orc_particle* q)
{
    memset(q, 0, sizeof(*q));
    q->E = p->E0;
    q->alive = 1;
    q->need_xs = 1;
    if (p->geometry == ORC_GEOM_SLAB) {
        q->u = 1.0;
        orc_set_region(p, q);
        return;
    }
    if (p->geometry == ORC_GEOM_LATTICE) {
        int32_t n = p->lattice_n;
        int64_t n2 = (int64_t)n * n;
        int64_t pin = (int64_t)(orc_draw(r) * (double)n2);
        if (pin >= n2) pin = n2 - 1;
        q->ci = (int32_t)(pin / n);
        q->cj = (int32_t)(pin % n);
        double half = 0.5 * (double)n * p->pitch;
        q->x = -half + p->pitch * ((double)q->ci + 0.5);
        q->y = -half + p->pitch * ((double)q->cj + 0.5);
        q->z = 0.5 * p->height;
        q->inpin = 1;
    }
    double mu = 2.0 * orc_draw(r) - 1.0;
    double c, s;
    orc_azimuth(r, &c, &s);
    double st = sqrt(1.0 - mu * mu);
    q->u = st * c;
    q->v = st * s;
    q->w = mu;
    orc_set_region(p, q);
}

/* Fission-spectrum energy: the Maxwellian chi(E) ~ sqrt(E) exp(-E/T), a
 * Gamma(3/2, T) variate, sampled as the sum of a Gamma(1) and a Gamma(1/2)
 * variate: E = -T (ln xi1 + ln xi2 cos^2 phi) with phi uniform (the
 * Box-Muller square of a normal; Everett and Cashwell's Monte Carlo sampler,
 * rule C64).  cos phi comes from the same disc rejection as the azimuth. */
static double orc_fission_energy(orc_rng* r, double T)
{
    double xi1 = orc_draw(r), xi2 = orc_draw(r);
    double c, s;
    orc_azimuth(r, &c, &s);
    return -T * (log(xi1) + (c * c) * log(xi2));
}

/* A history started from a fission site: the site's position and cell,
 * isotropic direction (mu, then azimuth), energy from the fission spectrum. */
static void orc_site_source(const orc_problem* p, orc_rng* r, const orc_site* st, double T,
                            orc_particle* q)
{
    memset(q, 0, sizeof(*q));
    q->alive = 1;
    q->need_xs = 1;
    q->x = st->x;
    q->y = st->y;
    q->z = st->z;
    q->ci = st->ci;
    q->cj = st->cj;
    q->inpin = st->inpin;
    double mu = 2.0 * orc_draw(r) - 1.0;
    double c, s;
    orc_azimuth(r, &c, &s);
    double sn = sqrt(1.0 - mu * mu);
    q->u = sn * c;
    q->v = sn * s;
    q->w = mu;
    q->E = orc_fission_energy(r, T);
    orc_set_region(p, q);
}

/* Distance to the nearest surface along the flight direction.  Candidates are
 * compared in a fixed order with strict '<', so earlier candidates win ties. */
static double orc_distance(const orc_problem* p, const orc_particle* q, int* surf)
{
    double d = INFINITY;
    *surf = ORC_S_NONE;
    if (p->geometry == ORC_GEOM_INFINITE) return d;
    if (p->geometry == ORC_GEOM_SLAB) {
        if (q->u > 0.0) {
            d = (p->slab_length - q->x) / q->u;
            *surf = ORC_S_XHI;
        } else if (q->u < 0.0) {
            d = (0.0 - q->x) / q->u;
            *surf = ORC_S_XLO;
        }
        if (d < 0.0) d = 0.0;
        return d;
    }
    /* lattice */
    if (q->w > 0.0) {
        d = (p->height - q->z) / q->w;
        *surf = ORC_S_ZTOP;
    } else if (q->w < 0.0) {
        d = (0.0 - q->z) / q->w;
        *surf = ORC_S_ZBOT;
    }
    int32_t n = p->lattice_n;
    double half = 0.5 * (double)n * p->pitch;
    double cx = -half + p->pitch * ((double)q->ci + 0.5);
    double cy = -half + p->pitch * ((double)q->cj + 0.5);
    double dx = q->x - cx, dy = q->y - cy;
    double a = q->u * q->u + q->v * q->v;
    double k = dx * q->u + dy * q->v;
    double c = dx * dx + dy * dy - p->radius * p->radius;
    double dc = INFINITY;
    if (q->inpin) {
        if (a > 0.0) {
            double disc = k * k - a * c;
            if (disc < 0.0) disc = 0.0;
            dc = (-k + sqrt(disc)) / a;
        }
    } else if (a > 0.0 && k < 0.0) {
        double disc = k * k - a * c;
        if (disc >= 0.0) dc = (-k - sqrt(disc)) / a;
    }
    if (dc < d) {
        d = dc;
        *surf = ORC_S_CYL;
    }
    if (!q->inpin) {
        double xl = -half + p->pitch * (double)q->ci;
        double xh = -half + p->pitch * (double)(q->ci + 1);
        double yl = -half + p->pitch * (double)q->cj;
        double yh = -half + p->pitch * (double)(q->cj + 1);
        if (q->u > 0.0) {
            double t = (xh - q->x) / q->u;
            if (t < d) { d = t; *surf = ORC_S_XHI; }
        } else if (q->u < 0.0) {
            double t = (xl - q->x) / q->u;
            if (t < d) { d = t; *surf = ORC_S_XLO; }
        }
        if (q->v > 0.0) {
            double t = (yh - q->y) / q->v;
            if (t < d) { d = t; *surf = ORC_S_YHI; }
        } else if (q->v < 0.0) {
            double t = (yl - q->y) / q->v;
            if (t < d) { d = t; *surf = ORC_S_YLO; }
        }
    }
    if (d < 0.0) d = 0.0;
    return d;
}

/* Logical surface crossing.  Returns the outcome index if the particle
 * leaves the problem, else -1. */
static int orc_cross(const orc_problem* p, orc_particle* q, int surf)
{
    int32_t n = p->lattice_n;
    switch (surf) {
    case ORC_S_ZTOP:
    case ORC_S_ZBOT:
        q->w = -q->w;
        return -1;
    case ORC_S_CYL:
        q->inpin = !q->inpin;
        break;
    case ORC_S_XHI:
        if (p->geometry == ORC_GEOM_SLAB || q->ci == n - 1) return ORC_OUT_LEAK_XHI;
        q->ci += 1;
        break;
    case ORC_S_XLO:
        if (p->geometry == ORC_GEOM_SLAB || q->ci == 0) return ORC_OUT_LEAK_OTHER;
        q->ci -= 1;
        break;
    case ORC_S_YHI:
        if (q->cj == n - 1) return ORC_OUT_LEAK_OTHER;
        q->cj += 1;
        break;
    case ORC_S_YLO:
        if (q->cj == 0) return ORC_OUT_LEAK_OTHER;
        q->cj -= 1;
        break;
    default:
        return ORC_OUT_LEAK_OTHER;
    }
    int32_t old_m = q->material;
    orc_set_region(p, q);
    if (q->material != old_m) q->need_xs = 1;
    return -1;
}

/* Direction rotation by the scattering cosine mu and azimuth (c, s), with the
 * alternative frame when |w| is close to 1. */
static void orc_rotate(orc_particle* q, double mu, double c, double s)
{
    double u = q->u, v = q->v, w = q->w;
    double a = sqrt(1.0 - mu * mu);
    if (fabs(w) < 0.9999) {
        double b = sqrt(1.0 - w * w);
        q->u = mu * u + a * (u * w * c - v * s) / b;
        q->v = mu * v + a * (v * w * c + u * s) / b;
        q->w = mu * w - a * b * c;
    } else {
        double b = sqrt(1.0 - v * v);
        q->u = mu * u + a * (u * v * c + w * s) / b;
        q->v = mu * v - a * b * c;
        q->w = mu * w + a * (v * w * c - u * s) / b;
    }
}

/* Collision (analog): species j = the first with xi1 * Sigma_t < C_j, C_j the
 * sequential cumulative sum of N_i (sigma_s,i + sigma_a,i) (the last species
 * if none qualifies); absorption if xi2 * sigma_t,j < sigma_a,j; otherwise
 * elastic scattering, isotropic in the centre-of-mass frame.  Returns the
 * outcome index if the particle dies, else -1.
 * Eigenvalue runs draw a fourth uniform xi4 and, before the reaction is
 * decided, bank floor(nuSigma_f / Sigma_t / k_norm + xi4) fission sites at
 * the collision point (the expected number of fission neutrons of the
 * collision, renormalised by the previous generation's k, rounded
 * stochastically); the collision scores nuSigma_f / Sigma_t to k. */
static int orc_collide(const orc_problem* p, orc_rng* r, orc_particle* q, orc_eigen* eig)
{
    double xi1 = orc_draw(r), xi2 = orc_draw(r), xi3 = orc_draw(r);
    if (eig) {
        double xi4 = orc_draw(r);
        double yield = q->sig_nf / q->sig_t;
        eig->k_col += yield;
        int64_t n_new = (int64_t)floor(yield / eig->k_norm + xi4);
        for (int64_t k = 0; k < n_new; ++k) {
            if (eig->n_sites == eig->cap_sites) {
                int64_t nc = eig->cap_sites ? 2 * eig->cap_sites : 8;
                orc_site* ns = (orc_site*)realloc(eig->sites, (size_t)nc * sizeof(orc_site));
                if (!ns) {
                    eig->failed = 1;
                    break;
                }
                eig->sites = ns;
                eig->cap_sites = nc;
            }
            orc_site* st = &eig->sites[eig->n_sites++];
            st->x = q->x;
            st->y = q->y;
            st->z = q->z;
            st->ci = q->ci;
            st->cj = q->cj;
            st->inpin = q->inpin;
        }
    }
    int32_t m = q->material;
    double target = xi1 * q->sig_t;
    double cum = 0.0, ss_j = 0.0, sa_j = 0.0;
    int32_t j = -1;
    for (int32_t i = p->mat_offsets[m]; i < p->mat_offsets[m + 1]; ++i) {
        int32_t s = p->mat_species[i];
        const double* g = p->energies + p->grid_offsets[s];
        int64_t np = p->grid_offsets[s + 1] - p->grid_offsets[s];
        const double* tab = p->sigma + p->grid_offsets[s] * p->n_ch;
        int64_t k = orc_grid_index(g, np, q->E);
        double f = orc_fraction(g, k, q->E);
        double s0 = tab[k * p->n_ch + p->ch_scatter], s1 = tab[(k + 1) * p->n_ch + p->ch_scatter];
        double a0 = tab[k * p->n_ch + p->ch_absorb], a1 = tab[(k + 1) * p->n_ch + p->ch_absorb];
        ss_j = s0 + f * (s1 - s0);
        sa_j = a0 + f * (a1 - a0);
        j = s;
        cum = cum + p->mat_dens[i] * (ss_j + sa_j);
        if (target < cum) break;
    }
    double st_j = ss_j + sa_j;
    if (xi2 * st_j < sa_j) return ORC_OUT_ABSORBED;
    double A = p->awr[j];
    double mu = 2.0 * xi3 - 1.0;
    double num = A * A + 2.0 * A * mu + 1.0;
    double den = (A + 1.0) * (A + 1.0);
    double E_new = q->E * (num / den);
    if (E_new < p->E_cut) return ORC_OUT_CUTOFF;
    double mu_lab = (1.0 + A * mu) / sqrt(num);
    if (mu_lab > 1.0) mu_lab = 1.0;
    if (mu_lab < -1.0) mu_lab = -1.0;
    double c, s;
    orc_azimuth(r, &c, &s);
    orc_rotate(q, mu_lab, c, s);
    q->E = E_new;
    q->need_xs = 1;
    return -1;
}

/* One history, start to end, scoring into batch b.  Returns 0, or -1 if the
 * per-history event cap was reached (the history is then abandoned without a
 * terminal score).  eig != NULL: an eigenvalue-run history (see orc_collide). */
static int orc_history(const orc_problem* p, orc_tallies* t, uint64_t seed, int64_t h, int64_t b,
                       uint32_t* ncoll_out, orc_eigen* eig)
{
    int32_t nb = orc_n_bins(p), M = p->n_materials;
    orc_rng r;
    orc_rng_init(&r, seed, p->problem_id, (uint64_t)h);
    orc_particle q;
    if (eig && eig->src)
        orc_site_source(p, &r, eig->src, eig->T, &q);
    else
        orc_source(p, &r, &q);
    int outcome = -1;
    for (int64_t ev = 0; ev < ORC_MAX_EVENTS_PER_HISTORY; ++ev) {
        if (q.need_xs) {
            orc_macro(p, q.material, q.E, &q.sig_t, &q.sig_a, eig ? &q.sig_nf : NULL);
            q.need_xs = 0;
        }
        double xi = orc_draw(&r);
        double dcol = q.sig_t > 0.0 ? -log(xi) / q.sig_t : INFINITY;
        int surf;
        double dsurf = orc_distance(p, &q, &surf);
        int collide = !(dsurf <= dcol);
        double d = collide ? dcol : dsurf;
        if (isinf(d)) {
            outcome = ORC_OUT_LEAK_OTHER;
            break;
        }
        q.x = q.x + d * q.u;
        q.y = q.y + d * q.v;
        q.z = q.z + d * q.w;
        int32_t bin = p->geometry == ORC_GEOM_INFINITE
                          ? (int32_t)orc_grid_index(p->ebin_edges, p->n_ebins + 1, q.E)
                          : q.region;
        double x_abs = d * q.sig_a;
        if (eig) eig->k_tl += d * q.sig_nf;
        t->flux[b * nb + bin] += d;
        t->absorb[b * nb + bin] += x_abs;
        if (p->derivatives) {
            int32_t m = q.material;
            q.W[m] = q.W[m] - q.sig_t * d;
            if (collide) q.W[m] = q.W[m] + 1.0;
            for (int32_t mm = 0; mm < M; ++mm) {
                t->dflux[(b * nb + bin) * M + mm] += d * q.W[mm];
                t->dabsorb[(b * nb + bin) * M + mm] += x_abs * q.W[mm] + (mm == m ? x_abs : 0.0);
            }
        }
        if (!collide) {
            int o = orc_cross(p, &q, surf);
            if (o >= 0) {
                outcome = o;
                break;
            }
        } else {
            q.ncoll += 1;
            t->outcome[b * ORC_N_OUT + ORC_OUT_COLLISIONS] += 1.0;
            if (p->derivatives)
                for (int32_t mm = 0; mm < M; ++mm)
                    t->doutcome[(b * ORC_N_OUT + ORC_OUT_COLLISIONS) * M + mm] += q.W[mm];
            int o = orc_collide(p, &r, &q, eig);
            if (o >= 0) {
                outcome = o;
                break;
            }
        }
    }
    if (ncoll_out) *ncoll_out = q.ncoll;
    if (outcome < 0) return -1;
    t->outcome[b * ORC_N_OUT + outcome] += 1.0;
    if (p->derivatives)
        for (int32_t mm = 0; mm < M; ++mm) t->doutcome[(b * ORC_N_OUT + outcome) * M + mm] += q.W[mm];
    return 0;
}

/* Runs histories [first, first + count) of the problem and adds their scores
 * to the tallies (which the caller zeroes).  Returns the number of histories
 * that hit the event cap (0 in a valid run), or -1 on a bad argument.
 * With n_threads > 1 histories run in parallel with private tallies that are
 * summed in thread order afterwards. */
int64_t orc_transport(const orc_problem* p, orc_tallies* t, int64_t first, int64_t count,
                      uint64_t seed, int n_threads)
{
    if (p->n_materials > ORC_MAX_DMAT && p->derivatives) return -1;
    if (first < 0 || count < 0 || first + count > p->n_histories_total) return -1;
    int32_t nb = orc_n_bins(p), M = p->n_materials;
    int64_t B = p->n_batches;
    size_t n_tal = (size_t)(B * nb), n_out = (size_t)(B * ORC_N_OUT);
    int64_t capped = 0;
    if (n_threads <= 1) {
        for (int64_t h = first; h < first + count; ++h)
            if (orc_history(p, t, seed, h, (h * B) / p->n_histories_total,
                            t->ncoll ? &t->ncoll[h - first] : NULL, NULL))
                capped++;
        return capped;
    }
#ifdef _OPENMP
    omp_set_num_threads(n_threads);
    int nt = n_threads;
    size_t per = 2 * n_tal + n_out + (p->derivatives ? (2 * n_tal + n_out) * M : 0);
    double* priv = (double*)calloc((size_t)nt * per, sizeof(double));
    if (!priv) return -1;
#pragma omp parallel reduction(+ : capped)
    {
        int tid = omp_get_thread_num();
        double* base = priv + (size_t)tid * per;
        orc_tallies mine;
        mine.flux = base;
        mine.absorb = base + n_tal;
        mine.outcome = base + 2 * n_tal;
        mine.dflux = p->derivatives ? base + 2 * n_tal + n_out : NULL;
        mine.dabsorb = p->derivatives ? mine.dflux + n_tal * M : NULL;
        mine.doutcome = p->derivatives ? mine.dabsorb + n_tal * M : NULL;
        mine.ncoll = NULL;
#pragma omp for schedule(dynamic, 64)
        for (int64_t h = first; h < first + count; ++h)
            if (orc_history(p, &mine, seed, h, (h * B) / p->n_histories_total,
                            t->ncoll ? &t->ncoll[h - first] : NULL, NULL))
                capped++;
    }
    for (int tid = 0; tid < nt; ++tid) {
        double* base = priv + (size_t)tid * per;
        for (size_t i = 0; i < n_tal; ++i) {
            t->flux[i] += base[i];
            t->absorb[i] += base[n_tal + i];
        }
        for (size_t i = 0; i < n_out; ++i) t->outcome[i] += base[2 * n_tal + i];
        if (p->derivatives) {
            double* d = base + 2 * n_tal + n_out;
            for (size_t i = 0; i < n_tal * M; ++i) {
                t->dflux[i] += d[i];
                t->dabsorb[i] += d[n_tal * M + i];
            }
            for (size_t i = 0; i < n_out * M; ++i) t->doutcome[i] += d[2 * n_tal * M + i];
        }
    }
    free(priv);
#else
    for (int64_t h = first; h < first + count; ++h)
        if (orc_history(p, t, seed, h, (h * B) / p->n_histories_total,
                        t->ncoll ? &t->ncoll[h - first] : NULL, NULL))
            capped++;
#endif
    return capped;
}

/* ------------------------------------------------------------------------ */
/* k-eigenvalue power iteration                                               */
/* ------------------------------------------------------------------------ */
/* Generation g runs N histories with ids g N .. g N + N - 1 (their own Philox
 * streams).  Generation 0 starts from the fixed source; generation g > 0
 * starts history g N + i from site i of its source, which is the previous
 * generation's bank resampled to N sites by the systematic selection
 * source[i] = bank[floor(i M / N)] (M banked sites, bank in the order of the
 * parent history and, within a history, of banking).  The site-count k of
 * generation g is k_g = M_g k_norm,g / N with k_norm,0 = k0 and
 * k_norm,g+1 = k_g; the collision and track-length estimators are the sums of
 * nuSigma_f / Sigma_t over collisions and of d nuSigma_f over flights, over
 * N.  Tallies score only in the last n_active generations: active history
 * j = (g - n_inactive) N + i falls in batch floor(j B / (n_active N)).
 * gen_out[g] = {k_g, k_col,g, k_tl,g, M_g}.  last_bank (optional) receives
 * the last generation's bank, up to bank_cap sites, as rows
 * {x, y, z, ci, cj, inpin}; *bank_n its size.  last_source (optional, N
 * rows of the same form) receives the sites the last generation started from
 * (none for a one-generation run).  ncoll (optional): collision counts of the
 * last generation's histories.
 * Returns 0; -1 bad arguments; -2 a generation banked no site; -3 out of
 * memory; -4 a history hit the event cap. */
int orc_eigenvalue(const orc_problem* p, orc_tallies* t, uint64_t seed, int64_t N,
                   int32_t n_generations, int32_t n_inactive, double k0, double T, int n_threads,
                   double* gen_out, double* last_bank, int64_t bank_cap, int64_t* bank_n,
                   double* last_source, uint32_t* ncoll)
{
    if (N < 1 || n_generations < 1 || n_inactive < 0 || n_inactive >= n_generations || !(k0 > 0.0) ||
        !(T > 0.0) || p->ch_nu_fission < 0 || p->ch_nu_fission >= p->n_ch || p->derivatives)
        return -1;
    int32_t nb = orc_n_bins(p);
    int64_t B = p->n_batches, n_active = n_generations - n_inactive;
    size_t n_tal = (size_t)(B * nb), n_out = (size_t)(B * ORC_N_OUT);
    double* scratch = (double*)calloc(2 * n_tal + n_out, sizeof(double));
    orc_eigen* hist = (orc_eigen*)calloc((size_t)N, sizeof(orc_eigen));
    orc_site* src = NULL;
    int rc = 0;
    if (!scratch || !hist) rc = -3;
    orc_tallies dump;
    memset(&dump, 0, sizeof(dump));
    dump.flux = scratch;
    dump.absorb = scratch ? scratch + n_tal : NULL;
    dump.outcome = scratch ? scratch + 2 * n_tal : NULL;
    double k_norm = k0;
#ifdef _OPENMP
    if (n_threads > 1) omp_set_num_threads(n_threads);
#endif
    for (int32_t g = 0; g < n_generations && rc == 0; ++g) {
        int active = g >= n_inactive;
        for (int64_t i = 0; i < N; ++i) {
            hist[i].k_norm = k_norm;
            hist[i].T = T;
            hist[i].src = src ? &src[i] : NULL;
            hist[i].n_sites = 0;
            hist[i].k_col = 0.0;
            hist[i].k_tl = 0.0;
        }
        int capped = 0;
        int last = g == n_generations - 1;
        if (last && last_source && src)
            for (int64_t i = 0; i < N; ++i) {
                double* row = last_source + 6 * i;
                row[0] = src[i].x;
                row[1] = src[i].y;
                row[2] = src[i].z;
                row[3] = (double)src[i].ci;
                row[4] = (double)src[i].cj;
                row[5] = (double)src[i].inpin;
            }
        /* tallies: the active generations into t (private per thread, summed
         * in thread order), the inactive ones into a scratch that is dropped */
        int nt = 1;
#ifdef _OPENMP
        nt = n_threads > 1 ? n_threads : 1;
#endif
        size_t per = 2 * n_tal + n_out;
        double* priv = (double*)calloc((size_t)nt * per, sizeof(double));
        if (!priv) {
            rc = -3;
            break;
        }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) reduction(| : capped)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            orc_tallies mine;
            memset(&mine, 0, sizeof(mine));
            mine.flux = priv + (size_t)tid * per;
            mine.absorb = mine.flux + n_tal;
            mine.outcome = mine.flux + 2 * n_tal;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t i = 0; i < N; ++i) {
                int64_t j = active ? (int64_t)(g - n_inactive) * N + i : 0;
                int64_t b = active ? (j * B) / (n_active * N) : 0;
                if (orc_history(p, &mine, seed, (int64_t)g * N + i, b,
                                (last && ncoll) ? &ncoll[i] : NULL, &hist[i]))
                    capped |= 1;
            }
        }
        orc_tallies* dst = active ? t : &dump;
        for (int tid = 0; tid < nt; ++tid) {
            double* base = priv + (size_t)tid * per;
            for (size_t i = 0; i < n_tal; ++i) {
                dst->flux[i] += base[i];
                dst->absorb[i] += base[n_tal + i];
            }
            for (size_t i = 0; i < n_out; ++i) dst->outcome[i] += base[2 * n_tal + i];
        }
        free(priv);
        if (capped) {
            rc = -4;
            break;
        }
        /* the bank in parent-history order, the estimators summed in that order */
        int64_t M = 0;
        double kc = 0.0, kt = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            if (hist[i].failed) rc = -3;
            M += hist[i].n_sites;
            kc += hist[i].k_col;
            kt += hist[i].k_tl;
        }
        if (rc) break;
        double k_g = ((double)M * k_norm) / (double)N;
        gen_out[4 * g + 0] = k_g;
        gen_out[4 * g + 1] = kc / (double)N;
        gen_out[4 * g + 2] = kt / (double)N;
        gen_out[4 * g + 3] = (double)M;
        if (M == 0) {
            rc = -2;
            break;
        }
        orc_site* bank = (orc_site*)malloc((size_t)M * sizeof(orc_site));
        orc_site* next = (orc_site*)malloc((size_t)N * sizeof(orc_site));
        if (!bank || !next) {
            free(bank);
            free(next);
            rc = -3;
            break;
        }
        int64_t pos = 0;
        for (int64_t i = 0; i < N; ++i)
            for (int64_t k = 0; k < hist[i].n_sites; ++k) bank[pos++] = hist[i].sites[k];
        if (last) {
            if (bank_n) *bank_n = M;
            if (last_bank)
                for (int64_t k = 0; k < M && k < bank_cap; ++k) {
                    double* row = last_bank + 6 * k;
                    row[0] = bank[k].x;
                    row[1] = bank[k].y;
                    row[2] = bank[k].z;
                    row[3] = (double)bank[k].ci;
                    row[4] = (double)bank[k].cj;
                    row[5] = (double)bank[k].inpin;
                }
        }
        for (int64_t i = 0; i < N; ++i) next[i] = bank[(i * M) / N];
        free(bank);
        free(src);
        src = next;
        k_norm = k_g;
    }
    for (int64_t i = 0; hist && i < N; ++i) free(hist[i].sites);
    free(hist);
    free(src);
    free(scratch);
    return rc;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Small exported wrappers so tests can pin single steps of the transport.    */
/* ------------------------------------------------------------------------ */

/* Elastic kinematics for mass ratio A and centre-of-mass cosine mu:
 * out[0] = E'/E, out[1] = the laboratory cosine (unclamped). */
void orc_scatter_kinematics(double A, double mu, double* out)
{
    double num = A * A + 2.0 * A * mu + 1.0;
    double den = (A + 1.0) * (A + 1.0);
    out[0] = num / den;
    out[1] = (1.0 + A * mu) / sqrt(num);
}

/* Rotate direction dir[3] by cosine mu and azimuth (c, s); result in out[3]. */
void orc_rotate_direction(const double* dir, double mu, double c, double s, double* out)
{
    orc_particle q;
    memset(&q, 0, sizeof(q));
    q.u = dir[0]; q.v = dir[1]; q.w = dir[2];
    orc_rotate(&q, mu, c, s);
    out[0] = q.u; out[1] = q.v; out[2] = q.w;
}

/* Source state of history h: out = {x, y, z, u, v, w, region, draws used}. */
void orc_source_state(const orc_problem* p, uint64_t seed, int64_t h, double* out)
{
    orc_rng r;
    orc_particle q;
    orc_rng_init(&r, seed, p->problem_id, (uint64_t)h);
    orc_source(p, &r, &q);
    out[0] = q.x; out[1] = q.y; out[2] = q.z;
    out[3] = q.u; out[4] = q.v; out[5] = q.w;
    out[6] = (double)q.region;
    out[7] = (double)r.n;
}

/* State {x, y, z, u, v, w, E, region, draws used} of history h started from
 * the fission site {x, y, z, ci, cj, inpin} (pins). */
void orc_site_source_state(const orc_problem* p, uint64_t seed, int64_t h, const double* site,
                           double T, double* out)
{
    orc_rng r;
    orc_particle q;
    orc_site st;
    st.x = site[0];
    st.y = site[1];
    st.z = site[2];
    st.ci = (int32_t)site[3];
    st.cj = (int32_t)site[4];
    st.inpin = (int32_t)site[5];
    orc_rng_init(&r, seed, p->problem_id, (uint64_t)h);
    orc_site_source(p, &r, &st, T, &q);
    out[0] = q.x; out[1] = q.y; out[2] = q.z;
    out[3] = q.u; out[4] = q.v; out[5] = q.w;
    out[6] = q.E;
    out[7] = (double)q.region;
    out[8] = (double)r.n;
}

/* Distance to the nearest surface from state st = {x, y, z, u, v, w, ci, cj,
 * inpin}; returns the surface id (ORC_S_*) and writes the distance. */
int orc_surface_distance(const orc_problem* p, const double* st, double* dist)
{
    orc_particle q;
    memset(&q, 0, sizeof(q));
    q.x = st[0]; q.y = st[1]; q.z = st[2];
    q.u = st[3]; q.v = st[4]; q.w = st[5];
    q.ci = (int32_t)st[6]; q.cj = (int32_t)st[7]; q.inpin = (int32_t)st[8];
    int surf;
    *dist = orc_distance(p, &q, &surf);
    return surf;
}

/* n successive fission-spectrum energies from history hist's stream (pins). */
void orc_fission_energies(uint64_t seed, uint32_t problem_id, uint64_t hist, double T, int64_t n,
                          double* out)
{
    orc_rng r;
    orc_rng_init(&r, seed, problem_id, hist);
    for (int64_t i = 0; i < n; ++i) out[i] = orc_fission_energy(&r, T);
}
