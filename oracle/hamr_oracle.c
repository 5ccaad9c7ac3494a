/*
 * hamr_oracle.c -- plain FP64 CPU oracle for the stochastic Landau-Lifshitz-Gilbert
 * (sLLG) Heun step on an atomistic spin lattice (arXiv 2502.02236, Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU library computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and it never imports it.
 *
 * What it computes, per Heun step n (t_n = n dt), stage by stage over all sites:
 *   1. local laser temperature T_i(t_n) (Gaussian spot, Sec. III / Fig. 2) and the
 *      thermal-field standard deviation sigma_i = sqrt(2 alpha kB T_i / (gamma mu_s dt))
 *      (Sec. II, text under Eq. 1, written in tesla: B = mu0 H);
 *   2. three standard normals xi_i from Philox4x32-10 (Salmon et al., SC'11) with
 *      key = replica seed, counter = (site, step), via Box-Muller;
 *   3. the effective field B_i(S) = (1/mu_s) sum_j J_ij S_j            (Eq. 2)
 *                                  + (2 ku / mu_s)(S_i . z) z          (Eq. 3)
 *                                  + B_app(t_n)                         (write field)
 *      plus B_th,i = sigma_i xi_i;
 *   4. predictor S'_i = N(S_i + dt f(S_i, B_i(S) + B_th,i)),
 *      f(S, B) = -gamma/(1+alpha^2) [S x B + alpha S x (S x B)]  (Eq. 1 in explicit
 *      Landau-Lifshitz form), N(v) = v/|v|;
 *   5. B_i(S') with the same xi and the same B_app(t_n);
 *   6. corrector S_i <- N(S_i + dt/2 [f(S_i, B_i(S)+B_th) + f(S'_i, B_i(S')+B_th)]).
 * Reductions: magnetisation M = sum S_i / N_mag and per-grain sums (Eq. 6 as an
 * average), energy E = -sum_pairs J_ij S_i.S_j - sum ku S_z^2 - sum mu_s B_app.S.
 *
 * The neighbour list is built from geometry alone: every lattice offset whose length
 * equals one of the shell distances (relative tolerance 1e-6) is a bond, wrapped on
 * periodic axes, dropped across open edges, and kept only when both ends carry the
 * same non-negative grain id (exchange-decoupled grains, Sec. II).  For the simple
 * cubic lattice this gives the 6 nearest neighbours; for the L1_0 Fe sublattice
 * (tetragonal a' = a/sqrt2, c) the 4 in-plane nearest, 2 out-of-plane and 4 in-plane
 * diagonal neighbours (Sec. II, Appendix A).
 */
#include "hamr_oracle.h"

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the round
 * multipliers 0xD2511F53 and 0xCD9E8D57, and a Weyl key schedule with increments
 * 0x9E3779B9 and 0xBB67AE85. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (seed, site, step): key = (seed low word, seed high word),
 * counter = (site low, site high, step low, step high); u_k = (x_k + 1/2) 2^-32 lies in
 * (0, 1); Box-Muller on (u0, u1) gives two normals, on (u2, u3) the third. */
void orc_thermal_normals(uint64_t seed, uint64_t site, uint64_t step, double xi[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32), (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)x[k] + 0.5) * (1.0 / 4294967296.0);
    double r1 = sqrt(-2.0 * log(u[0]));
    double r2 = sqrt(-2.0 * log(u[2]));
    xi[0] = r1 * cos(2.0 * ORC_PI * u[1]);
    xi[1] = r1 * sin(2.0 * ORC_PI * u[1]);
    xi[2] = r2 * cos(2.0 * ORC_PI * u[3]);
}

/* ------------------------------------------------------------------------- */
/* Drivers (Sec. III, Fig. 2): Gaussian laser temperature and trapezoidal write field */

static void site_coords(const orc_params *p, int64_t i, int *ix, int *iy, int *iz)
{
    *ix = (int)(i % p->nx);
    *iy = (int)((i / p->nx) % p->ny);
    *iz = (int)(i / ((int64_t)p->nx * p->ny));
}

double orc_temperature(const orc_params *p, double x, double y, double t)
{
    if (!(p->fwhm > 0.0)) return p->T_amb;
    double dx = x - p->x0 - p->vx * t;
    double dy = y - p->y0 - p->vy * t;
    double r2 = dx * dx + dy * dy;
    return p->T_amb + (p->T_peak - p->T_amb) * exp(-4.0 * log(2.0) * r2 / (p->fwhm * p->fwhm));
}

static double bit_polarity(const orc_params *p, long b)
{
    if (b < 0) b = 0;
    if (b > p->n_bits - 1) b = p->n_bits - 1;
    return p->bits[b] ? -1.0 : 1.0;
}

/* Field polarity s(t) in [-1, 1]: the head at x_h = head_x0 + head_v t sits in bit
 * b = floor(x_h / bit_len); the polarity ramps linearly from bit b-1's to bit b's over
 * the first ramp_len of bit b and is flat afterwards. */
double orc_field_polarity(const orc_params *p, double t)
{
    if (p->n_bits <= 0) return 1.0;
    double xh = p->head_x0 + p->head_v * t;
    double fb = floor(xh / p->bit_len);
    long b = (long)fb;
    double into = xh - fb * p->bit_len;
    double prev = bit_polarity(p, b - 1), cur = bit_polarity(p, b);
    double w = (p->ramp_len > 0.0) ? into / p->ramp_len : 1.0;
    if (w > 1.0) w = 1.0;
    if (w < 0.0) w = 0.0;
    return prev + (cur - prev) * w;
}

void orc_applied_field(const orc_params *p, double t, double B[3])
{
    double s = orc_field_polarity(p, t);
    for (int d = 0; d < 3; ++d) B[d] = p->B0 * s * p->dir[d];
}

/* ------------------------------------------------------------------------- */
/* Neighbours from geometry */

static int wrap_or_reject(int v, int n, int periodic, int *out)
{
    if (v >= 0 && v < n) { *out = v; return 1; }
    if (!periodic) return 0;
    *out = ((v % n) + n) % n;
    return 1;
}

/* Bonds of site i: writes neighbour index and shell id, returns their number. */
int orc_site_neighbours(const orc_params *p, const int32_t *grain, int64_t i, int64_t *js, int32_t *shells, int cap)
{
    if (grain[i] < 0) return 0;
    double rmax = 0.0;
    for (int s = 0; s < p->n_shells; ++s) if (p->shell_dist[s] > rmax) rmax = p->shell_dist[s];
    int mx = (int)floor(rmax / p->ax * (1.0 + 1e-6));
    int my = (int)floor(rmax / p->ay * (1.0 + 1e-6));
    int mz = (int)floor(rmax / p->az * (1.0 + 1e-6));
    int ix, iy, iz;
    site_coords(p, i, &ix, &iy, &iz);
    int count = 0;
    for (int dk = -mz; dk <= mz; ++dk)
        for (int dj = -my; dj <= my; ++dj)
            for (int di = -mx; di <= mx; ++di) {
                if (di == 0 && dj == 0 && dk == 0) continue;
                double dx = di * p->ax, dy = dj * p->ay, dz = dk * p->az;
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                int shell = -1;
                for (int s = 0; s < p->n_shells; ++s)
                    if (fabs(d - p->shell_dist[s]) <= 1e-6 * p->shell_dist[s]) shell = s;
                if (shell < 0) continue;
                int jx, jy, jz;
                if (!wrap_or_reject(ix + di, p->nx, p->periodic[0], &jx)) continue;
                if (!wrap_or_reject(iy + dj, p->ny, p->periodic[1], &jy)) continue;
                if (!wrap_or_reject(iz + dk, p->nz, p->periodic[2], &jz)) continue;
                int64_t j = (int64_t)jx + (int64_t)p->nx * ((int64_t)jy + (int64_t)p->ny * jz);
                if (grain[j] != grain[i]) continue;
                if (count < cap) {
                    js[count] = j;
                    shells[count] = shell;
                }
                ++count;
            }
    return count;
}

/* ------------------------------------------------------------------------- */
/* Field and equation of motion */

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void normalise(double v[3])
{
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= r; v[1] /= r; v[2] /= r;
}

/* f(S, B) = -gamma/(1+alpha^2) [S x B + alpha S x (S x B)] */
void orc_llg_rhs(const orc_params *p, const double S[3], const double B[3], double f[3])
{
    double sxb[3], sxsxb[3];
    cross(S, B, sxb);
    cross(S, sxb, sxsxb);
    double pref = -p->gamma / (1.0 + p->alpha * p->alpha);
    for (int d = 0; d < 3; ++d) f[d] = pref * (sxb[d] + p->alpha * sxsxb[d]);
}

/* Deterministic part of the field at site i for spin configuration S (AoS [3n]). */
static void site_field(const orc_params *p, const double *S, int64_t i, int nb, const int64_t *js,
                       const int32_t *shells, const double Bapp[3], double B[3])
{
    double ex[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < nb; ++k) {
        const double *Sj = S + 3 * js[k];
        double Jk = p->J[shells[k]];
        ex[0] += Jk * Sj[0];
        ex[1] += Jk * Sj[1];
        ex[2] += Jk * Sj[2];
    }
    const double *Si = S + 3 * i;
    double ani = 2.0 * p->ku / p->mu_s * Si[2];
    B[0] = ex[0] / p->mu_s + Bapp[0];
    B[1] = ex[1] / p->mu_s + Bapp[1];
    B[2] = ex[2] / p->mu_s + ani + Bapp[2];
}

static void site_thermal_field(const orc_params *p, int64_t i, int64_t step, double Bth[3])
{
    int ix, iy, iz;
    site_coords(p, i, &ix, &iy, &iz);
    double t = (double)step * p->dt;
    double T = orc_temperature(p, (ix + 0.5) * p->ax, (iy + 0.5) * p->ay, t);
    double sigma = sqrt(2.0 * p->alpha * ORC_KB * T / (p->gamma * p->mu_s * p->dt));
    double xi[3];
    orc_thermal_normals(p->seed, (uint64_t)i, (uint64_t)step, xi);
    for (int d = 0; d < 3; ++d) Bth[d] = sigma * xi[d];
}

/* ------------------------------------------------------------------------- */
/* Context: parameters, grain map and the geometric neighbour list in CSR form */

typedef struct {
    orc_params p;
    uint8_t *bits;
    int64_t n;
    int32_t *grain;
    int64_t *row_ptr;   /* [n+1] */
    int64_t *col;       /* [nnz] */
    int32_t *shell;     /* [nnz] */
} orc_ctx;

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->bits);
    free(c->grain);
    free(c->row_ptr);
    free(c->col);
    free(c->shell);
    free(c);
}

orc_ctx *orc_create(const orc_params *p, const int32_t *grain)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->p = *p;
    if (p->n_bits > 0) {
        c->bits = (uint8_t *)malloc((size_t)p->n_bits);
        memcpy(c->bits, p->bits, (size_t)p->n_bits);
        c->p.bits = c->bits;
    }
    c->n = (int64_t)p->nx * p->ny * p->nz;
    c->grain = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->n);
    memcpy(c->grain, grain, sizeof(int32_t) * (size_t)c->n);
    c->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->n + 1));
    int64_t js[128];
    int32_t sh[128];
    c->row_ptr[0] = 0;
    for (int64_t i = 0; i < c->n; ++i)
        c->row_ptr[i + 1] = c->row_ptr[i] + orc_site_neighbours(&c->p, c->grain, i, js, sh, 128);
    int64_t nnz = c->row_ptr[c->n];
    c->col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    c->shell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        int64_t jj[128];
        int32_t ss[128];
        int nb = orc_site_neighbours(&c->p, c->grain, i, jj, ss, 128);
        for (int k = 0; k < nb; ++k) {
            c->col[c->row_ptr[i] + k] = jj[k];
            c->shell[c->row_ptr[i] + k] = ss[k];
        }
    }
    return c;
}

int64_t orc_n_sites(const orc_ctx *c) { return c->n; }
int64_t orc_nnz(const orc_ctx *c) { return c->row_ptr[c->n]; }

void orc_get_neighbours(const orc_ctx *c, int64_t *row_ptr, int64_t *col, int32_t *shell)
{
    memcpy(row_ptr, c->row_ptr, sizeof(int64_t) * (size_t)(c->n + 1));
    memcpy(col, c->col, sizeof(int64_t) * (size_t)c->row_ptr[c->n]);
    memcpy(shell, c->shell, sizeof(int32_t) * (size_t)c->row_ptr[c->n]);
}

/* Update the time-dependent drivers between step blocks. */
void orc_set_drivers(orc_ctx *c, double T_amb, double T_peak, double fwhm, double x0, double y0,
                     double vx, double vy)
{
    c->p.T_amb = T_amb; c->p.T_peak = T_peak; c->p.fwhm = fwhm;
    c->p.x0 = x0; c->p.y0 = y0; c->p.vx = vx; c->p.vy = vy;
}

/* One Heun step, stages 1-6 above, each a full pass over the lattice.  S is AoS [3n]
 * and is overwritten with the new state.  Returns 0, or -1 on allocation failure. */
int orc_heun_step(orc_ctx *c, double *S, int64_t step)
{
    const orc_params *p = &c->p;
    int64_t n = c->n;
    double *Bth = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *f1 = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *Sp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!Bth || !f1 || !Sp) {
        free(Bth); free(f1); free(Sp);
        return -1;
    }
    double Bapp[3];
    orc_applied_field(p, (double)step * p->dt, Bapp);

    /* 1-2: thermal field */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (c->grain[i] < 0) { Bth[3 * i] = Bth[3 * i + 1] = Bth[3 * i + 2] = 0.0; continue; }
        site_thermal_field(p, i, step, Bth + 3 * i);
    }
    /* 3-4: field at S, predictor */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (c->grain[i] < 0) {
            for (int d = 0; d < 3; ++d) { Sp[3 * i + d] = S[3 * i + d]; f1[3 * i + d] = 0.0; }
            continue;
        }
        int64_t r0 = c->row_ptr[i];
        int nb = (int)(c->row_ptr[i + 1] - r0);
        double B[3];
        site_field(p, S, i, nb, c->col + r0, c->shell + r0, Bapp, B);
        for (int d = 0; d < 3; ++d) B[d] += Bth[3 * i + d];
        orc_llg_rhs(p, S + 3 * i, B, f1 + 3 * i);
        for (int d = 0; d < 3; ++d) Sp[3 * i + d] = S[3 * i + d] + p->dt * f1[3 * i + d];
        normalise(Sp + 3 * i);
    }
    /* 5-6: field at S', corrector */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (c->grain[i] < 0) continue;
        int64_t r0 = c->row_ptr[i];
        int nb = (int)(c->row_ptr[i + 1] - r0);
        double B[3], f2[3];
        site_field(p, Sp, i, nb, c->col + r0, c->shell + r0, Bapp, B);
        for (int d = 0; d < 3; ++d) B[d] += Bth[3 * i + d];
        orc_llg_rhs(p, Sp + 3 * i, B, f2);
        for (int d = 0; d < 3; ++d) S[3 * i + d] = S[3 * i + d] + 0.5 * p->dt * (f1[3 * i + d] + f2[d]);
        normalise(S + 3 * i);
    }
    free(Bth); free(f1); free(Sp);
    return 0;
}

/* M = sum of S over magnetic sites / their number. */
void orc_magnetisation(const orc_ctx *c, const double *S, double M[3])
{
    double m[3] = {0.0, 0.0, 0.0};
    int64_t nmag = 0;
    for (int64_t i = 0; i < c->n; ++i) {
        if (c->grain[i] < 0) continue;
        for (int d = 0; d < 3; ++d) m[d] += S[3 * i + d];
        ++nmag;
    }
    for (int d = 0; d < 3; ++d) M[d] = nmag > 0 ? m[d] / (double)nmag : 0.0;
}

/* Run n_steps steps from step index step0; every record_every completed steps store M
 * into M_rec (3 doubles per record).  Returns the number of records, or -1. */
int64_t orc_run(orc_ctx *c, double *S, int64_t step0, int64_t n_steps, int32_t record_every, double *M_rec)
{
    int64_t nrec = 0;
    for (int64_t k = 0; k < n_steps; ++k) {
        if (orc_heun_step(c, S, step0 + k) != 0) return -1;
        if (record_every > 0 && (step0 + k + 1) % record_every == 0) {
            if (M_rec) orc_magnetisation(c, S, M_rec + 3 * nrec);
            ++nrec;
        }
    }
    return nrec;
}

/* Per-grain sums of S (Eq. 6 numerator) and site counts, grains 0..n_grains-1. */
void orc_grain_sums(const orc_ctx *c, const double *S, int32_t n_grains, double *sums, int64_t *counts)
{
    for (int32_t g = 0; g < n_grains; ++g) {
        sums[3 * g] = sums[3 * g + 1] = sums[3 * g + 2] = 0.0;
        counts[g] = 0;
    }
    for (int64_t i = 0; i < c->n; ++i) {
        int32_t g = c->grain[i];
        if (g < 0 || g >= n_grains) continue;
        for (int d = 0; d < 3; ++d) sums[3 * g + d] += S[3 * i + d];
        counts[g] += 1;
    }
}

/* E = -1/2 sum_i sum_j J_ij S_i.S_j - sum_i ku (S_i.z)^2 - sum_i mu_s B_app(t).S_i  [J] */
double orc_energy(const orc_ctx *c, const double *S, int64_t step)
{
    const orc_params *p = &c->p;
    double Bapp[3];
    orc_applied_field(p, (double)step * p->dt, Bapp);
    double E = 0.0;
    for (int64_t i = 0; i < c->n; ++i) {
        if (c->grain[i] < 0) continue;
        const double *Si = S + 3 * i;
        for (int64_t k = c->row_ptr[i]; k < c->row_ptr[i + 1]; ++k) {
            const double *Sj = S + 3 * c->col[k];
            E -= 0.5 * p->J[c->shell[k]] * (Si[0] * Sj[0] + Si[1] * Sj[1] + Si[2] * Sj[2]);
        }
        E -= p->ku * Si[2] * Si[2];
        E -= p->mu_s * (Bapp[0] * Si[0] + Bapp[1] * Si[1] + Bapp[2] * Si[2]);
    }
    return E;
}

/* The state after one step at selected sites only, from the full pre-step state S
 * (AoS [3n]); each requested site is computed from its own neighbourhood with the
 * same stages as orc_heun_step.  Used to check very large lattices one site at a time. */
int orc_step_sites(const orc_params *p, const int32_t *grain, const double *S, int64_t step,
                   int64_t n_sample, const int64_t *sites, double *S_out)
{
    double Bapp[3];
    orc_applied_field(p, (double)step * p->dt, Bapp);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int64_t q = 0; q < n_sample; ++q) {
        int64_t i = sites[q];
        double *out = S_out + 3 * q;
        if (grain[i] < 0) {
            for (int d = 0; d < 3; ++d) out[d] = S[3 * i + d];
            continue;
        }
        int64_t ji[128];
        int32_t si[128];
        int nbi = orc_site_neighbours(p, grain, i, ji, si, 128);
        if (nbi > 128) { ++bad; continue; }
        /* S' at i and at each neighbour of i, each from its own neighbourhood */
        double Spi[3], f1i[3], Bthi[3];
        double exn[3] = {0.0, 0.0, 0.0}; /* sum_j J_ij S'_j */
        for (int k = -1; k < nbi; ++k) {
            int64_t j = (k < 0) ? i : ji[k];
            int64_t jj[128];
            int32_t sj[128];
            int nbj = orc_site_neighbours(p, grain, j, jj, sj, 128);
            double B[3], Bth[3], f[3], Sp[3];
            site_field(p, S, j, nbj, jj, sj, Bapp, B);
            site_thermal_field(p, j, step, Bth);
            for (int d = 0; d < 3; ++d) B[d] += Bth[d];
            orc_llg_rhs(p, S + 3 * j, B, f);
            for (int d = 0; d < 3; ++d) Sp[d] = S[3 * j + d] + p->dt * f[d];
            normalise(Sp);
            if (k < 0) {
                for (int d = 0; d < 3; ++d) { Spi[d] = Sp[d]; f1i[d] = f[d]; Bthi[d] = Bth[d]; }
            } else {
                double Jk = p->J[si[k]];
                for (int d = 0; d < 3; ++d) exn[d] += Jk * Sp[d];
            }
        }
        double B2[3] = {exn[0] / p->mu_s + Bapp[0], exn[1] / p->mu_s + Bapp[1],
                        exn[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Spi[2] + Bapp[2]};
        for (int d = 0; d < 3; ++d) B2[d] += Bthi[d];
        double f2[3];
        orc_llg_rhs(p, Spi, B2, f2);
        for (int d = 0; d < 3; ++d) out[d] = S[3 * i + d] + 0.5 * p->dt * (f1i[d] + f2[d]);
        normalise(out);
    }
    return bad ? -1 : 0;
}
