/*
 * hamr_ms_oracle.c -- plain FP64 CPU oracle for the multiscale window of the paper
 * (Sec. II and Fig. 1): a simple-cubic atomistic window embedded in a micromagnetic
 * finite-difference track, exchange coupled across the interface and moving with the
 * laser spot.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU baseline may load it.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Geometry.  The track is ncx x ncy x ncz cubic cells of edge `cell`.  The atomistic
 * lattice has spacing a = cell / ratio, so each cell holds ratio^3 sites.  The window is
 * wx cells long, starts at cell column ox and spans every cell in y and z.  A cell's grain
 * id (-1 = non-magnetic) is shared by every site inside it.
 *
 * One coupled step n -> n+1 (t_n = n dt).  Drivers (laser temperature, write field) are
 * frozen at t_n for the whole step; the write field is uniform or follows the head with tanh
 * profiles along the track (orc_ms_field).  Optionally the demagnetising field of Eq. 7
 * (demag_stage, after stage 1) is added to the field of both regions, frozen for the step.
 *   1. Eq. 6: each cell inside the window takes the direction of the sum of its
 *      atomistic spins (0 for a non-magnetic cell).  The micromagnetic exchange of the
 *      neighbouring cells then sees the average atomistic direction (Sec. II).
 *   2. The atomistic sLLG Heun step of the window (Eq. 1-3, thermal field as in
 *      hamr_oracle.c, counter = the site's index on the whole track).  A site whose
 *      x-neighbour lies outside the window takes, for that bond, the direction of the
 *      micromagnetic cell containing the neighbour (Eq. 2 with the cell's m, Sec. II).
 *      Bonds join only sites (or a site and a cell) of the same grain.
 *   3. One classical RK4 step of the micromagnetic LLG (Eq. 1 without the thermal field)
 *      on every magnetic cell outside the window, with
 *        B = (2 A(T) / Ms(T)) lap(m) + (2 K(T) / Ms(T)) (m.z) z + B_app        (Eq. 4, 5)
 *      where lap is the 6-neighbour finite-difference Laplacian over same-grain magnetic
 *      neighbours (a missing neighbour adds nothing), Ms(T) = Ms0 m_e, A(T) = A0 m_e^2,
 *      K(T) = K0 m_e^3, damping alpha(T) = lambda (1 - T / 3 T_C) with T capped at T_C,
 *      and m_e(T) the root of m = L(3 T_C m / T + mu_s |B_app| / (kB T)) with the
 *      Langevin function L(x) = coth x - 1/x (Sec. II).  Cells inside the window are
 *      frozen at their Eq. 6 directions.  m is renormalised after the step.
 *   4. If the window follows the laser, it is moved forward one cell column at a time
 *      until it is centred on the spot (Sec. II, Fig. 1): the trailing column is handed to
 *      the micromagnetic side by Eq. 6, the sites shift back by `ratio`, and the new
 *      leading column is thermalised: every site gets a spin whose polar angle from the
 *      cell's m is uniform in [0, theta_max] and whose azimuth is uniform, with
 *      theta_max = (5 pi / 9) sqrt(1 - sqrt(1 + 6 (M/Ms0 - 1) / 5)) and M/Ms0 = m_e(T) of
 *      the cell (the square root's argument is kept in [0, 1]).
 */
#include "hamr_oracle.h"

typedef struct {
    int32_t ncx, ncy, ncz;  /* micromagnetic cells */
    double cell;            /* cell edge [m] */
    int32_t ratio;          /* atomistic sites per cell edge */
    int32_t wx;             /* window length in cells */
    double J, mu_s, ku;     /* atomistic exchange [J], moment [J/T], anisotropy per atom [J] */
    double Ms0, A0, K0;     /* micromagnetic Ms [A/m], A [J/m], K [J/m^3] at 0 K */
    double lambda;          /* atomistic damping; micromagnetic alpha(T) = lambda (1 - T/3T_C) */
    double T_C;             /* Curie temperature [K] */
    orc_params drv;         /* gamma, dt, seed, laser spot and write field (other fields unused) */
    int32_t profile;        /* 0: spatially uniform write field; 1: tanh profiles along the track */
    double prof_wz, prof_dz; /* width and offset from the head of the profile of B0 dir [m] */
    double prof_Bx0;        /* amplitude of the in-plane (x) component [T] */
    double prof_wx, prof_dx; /* its width and offset from the head [m] */
    int32_t demag;          /* 1: add the demagnetising field of Eq. 7 in both regions */
    int32_t margin;         /* < 0: every micromagnetic cell is evolved; >= 0: only the cells of the
                               simulated region, columns [ox - margin, ox + wx + margin), are; the
                               others are frozen (Sec. II, Fig. 1) */
} orc_ms_params;

typedef struct {
    orc_ms_params p;
    uint8_t *bits;
    int64_t nc;             /* cells */
    int32_t *grain;         /* [nc] */
    double *m;              /* [3 nc] AoS; window cells hold their Eq. 6 directions */
    int32_t ox;             /* first cell column of the window */
    int64_t nw;             /* sites in the window */
    double *S;              /* [3 nw] AoS, site (i, j, k) at i + nxw (j + nyw k) */
    int64_t step;           /* completed steps */
    int64_t events;         /* thermalisation events so far (window placements and moves) */
    int32_t live;           /* 1: the window's sites are newer than its cells (placed, and the
                               cells not replaced since) */
    double *Bd;             /* [3 nc] demagnetising field of the current step [T], or NULL */
    double *me_store;       /* [nc] m_e of each cell at its last evolved step (or the window's
                               placement): the m_e of a frozen cell */
} orc_ms;

/* ------------------------------------------------------------------------- */
/* Temperature dependence of the micromagnetic parameters (Sec. II) */

/* Langevin function coth x - 1/x; its series x/3 - x^3/45 + 2x^5/945 near 0. */
double orc_langevin(double x)
{
    if (fabs(x) < 1e-3) return x / 3.0 - x * x * x / 45.0 + 2.0 * x * x * x * x * x / 945.0;
    return 1.0 / tanh(x) - 1.0 / x;
}

/* m_e(T): the largest root in [0, 1] of m = L(3 T_C m / T + mu_s B / (kB T)), by
 * bisection on the sign of L(...) - m (m_e = 1 at T <= 0). */
double orc_me(double T_C, double T, double mu_s, double B)
{
    if (!(T > 0.0)) return 1.0;
    double a = 3.0 * T_C / T, b = mu_s * B / (ORC_KB * T);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_langevin(a * mid + b) - mid >= 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

double orc_ms_alpha(const orc_ms_params *p, double T)
{
    double Tc = T < p->T_C ? T : p->T_C;
    if (Tc < 0.0) Tc = 0.0;
    return p->lambda * (1.0 - Tc / (3.0 * p->T_C));
}

/* The cone half-angle of the thermalisation rule for M / Ms0 = mr. */
double orc_theta_max(double mr)
{
    double x = 1.0 + 6.0 * (mr - 1.0) / 5.0;
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    return (5.0 * ORC_PI / 9.0) * sqrt(1.0 - sqrt(x));
}

/* A unit spin in the cone of half-angle theta_max around the unit vector e3: polar angle
 * theta = u0 theta_max, azimuth phi = 2 pi u1 about e3, measured from
 * e1 = (z x e3)/|z x e3| (or (x x e3)/|x x e3| when |e3_z| >= 0.9), e2 = e3 x e1; u0 and
 * u1 are the first two words of Philox4x32-10 with key (seed low, seed high) and counter
 * (site low, site high, event low, event high | 2^31), mapped to (x + 1/2) 2^-32. */
void orc_cone_sample(const double e3[3], double theta_max, uint64_t seed, uint64_t site, uint64_t event,
                     double out[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32), (uint32_t)event,
                       (uint32_t)(event >> 32) | 0x80000000u};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u0 = ((double)x[0] + 0.5) * (1.0 / 4294967296.0);
    double u1 = ((double)x[1] + 0.5) * (1.0 / 4294967296.0);
    double th = u0 * theta_max, ph = 2.0 * ORC_PI * u1;
    double e1[3];
    if (fabs(e3[2]) < 0.9) {
        e1[0] = -e3[1]; e1[1] = e3[0]; e1[2] = 0.0;            /* z x e3 */
    } else {
        e1[0] = 0.0; e1[1] = -e3[2]; e1[2] = e3[1];            /* x x e3 */
    }
    double r = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int d = 0; d < 3; ++d) e1[d] /= r;
    double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    double a1 = sin(th) * cos(ph), a2 = sin(th) * sin(ph), a3 = cos(th);
    for (int d = 0; d < 3; ++d) out[d] = a1 * e1[d] + a2 * e2[d] + a3 * e3[d];
}

/* The write field at track position x and time t (Sec. III, Fig. 2).  Uniform: B0 s(t) dir.
 * With the head profile: each component is a tanh step along the track that follows the
 * head at x_h(t) = head_x0 + head_v t,
 *   B(x, t) = B0 s(t) dir P(x - x_h - dz, wz) + Bx0 s(t) P(x - x_h - dx, wx) x,
 *   P(u, w) = (1 - tanh(u / w)) / 2,
 * full under the pole upstream and zero downstream, with s(t) the bit polarity. */
void orc_ms_field(const orc_ms_params *p, double x, double t, double B[3])
{
    orc_applied_field(&p->drv, t, B);
    if (!p->profile) return;
    double s = orc_field_polarity(&p->drv, t);
    double xh = p->drv.head_x0 + p->drv.head_v * t;
    double Pz = 0.5 * (1.0 - tanh((x - xh - p->prof_dz) / p->prof_wz));
    double Px = 0.5 * (1.0 - tanh((x - xh - p->prof_dx) / p->prof_wx));
    for (int d = 0; d < 3; ++d) B[d] *= Pz;
    B[0] += p->prof_Bx0 * s * Px;
}

/* ------------------------------------------------------------------------- */
/* Context */

static int64_t cell_index(const orc_ms_params *p, int64_t cx, int64_t cy, int64_t cz)
{
    return cx + (int64_t)p->ncx * (cy + (int64_t)p->ncy * cz);
}

int64_t orc_ms_window_sites(const orc_ms_params *p)
{
    return (int64_t)p->wx * p->ratio * (int64_t)p->ncy * p->ratio * (int64_t)p->ncz * p->ratio;
}

void orc_ms_destroy(orc_ms *c)
{
    if (!c) return;
    free(c->bits); free(c->grain); free(c->m); free(c->S); free(c->Bd); free(c->me_store);
    free(c);
}

orc_ms *orc_ms_create(const orc_ms_params *p, const int32_t *cell_grain)
{
    orc_ms *c = (orc_ms *)calloc(1, sizeof(orc_ms));
    if (!c) return NULL;
    c->p = *p;
    if (p->drv.n_bits > 0) {
        c->bits = (uint8_t *)malloc((size_t)p->drv.n_bits);
        memcpy(c->bits, p->drv.bits, (size_t)p->drv.n_bits);
        c->p.drv.bits = c->bits;
    }
    c->nc = (int64_t)p->ncx * p->ncy * p->ncz;
    c->grain = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->nc);
    memcpy(c->grain, cell_grain, sizeof(int32_t) * (size_t)c->nc);
    c->m = (double *)calloc(3 * (size_t)c->nc, sizeof(double));
    c->nw = orc_ms_window_sites(p);
    c->S = (double *)calloc(3 * (size_t)c->nw, sizeof(double));
    c->Bd = (double *)calloc(3 * (size_t)c->nc, sizeof(double));
    c->me_store = (double *)calloc((size_t)c->nc, sizeof(double));
    if (!c->grain || !c->m || !c->S || !c->Bd || !c->me_store) {
        orc_ms_destroy(c);
        return NULL;
    }
    return c;
}

/* Replaces the drivers of a context between steps, as the library's setters do: the laser
 * spot, the write field with its bit pattern and head profile, and the switch of the
 * demagnetising field.  The step count, the window and the state stay.  A second pass along a
 * parallel track (Sec. III) is a new spot centre y0 and spot and head starting points for the
 * current time.  Returns -1, and changes nothing, when p describes another track, material,
 * time step or seed. */
int orc_ms_set_drivers(orc_ms *c, const orc_ms_params *p)
{
    const orc_ms_params *o = &c->p;
    if (p->ncx != o->ncx || p->ncy != o->ncy || p->ncz != o->ncz || p->cell != o->cell || p->ratio != o->ratio ||
        p->wx != o->wx || p->J != o->J || p->mu_s != o->mu_s || p->ku != o->ku || p->Ms0 != o->Ms0 ||
        p->A0 != o->A0 || p->K0 != o->K0 || p->lambda != o->lambda || p->T_C != o->T_C ||
        p->drv.dt != o->drv.dt || p->drv.gamma != o->drv.gamma || p->drv.seed != o->drv.seed)
        return -1;
    uint8_t *bits = NULL;
    if (p->drv.n_bits > 0) {
        bits = (uint8_t *)malloc((size_t)p->drv.n_bits);
        if (!bits) return -1;
        memcpy(bits, p->drv.bits, (size_t)p->drv.n_bits);
    }
    free(c->bits);
    c->bits = bits;
    c->p = *p;
    c->p.drv.bits = bits;
    return 0;
}

void orc_ms_set_cells(orc_ms *c, const double *m)
{
    for (int64_t q = 0; q < c->nc; ++q)
        for (int d = 0; d < 3; ++d) c->m[3 * q + d] = c->grain[q] >= 0 ? m[3 * q + d] : 0.0;
    c->live = 0;
}

void orc_ms_get_cells(const orc_ms *c, double *m) { memcpy(m, c->m, sizeof(double) * 3 * (size_t)c->nc); }
void orc_ms_get_moments(const orc_ms *c, double *S) { memcpy(S, c->S, sizeof(double) * 3 * (size_t)c->nw); }
void orc_ms_set_moments(orc_ms *c, const double *S) { memcpy(c->S, S, sizeof(double) * 3 * (size_t)c->nw); }
int32_t orc_ms_window(const orc_ms *c) { return c->ox; }
int64_t orc_ms_step_count(const orc_ms *c) { return c->step; }

/* Site (i, j, k) of the window: its cell, grain and index on the whole track. */
static int64_t site_cell(const orc_ms *c, int64_t i, int64_t j, int64_t k)
{
    const int r = c->p.ratio;
    return cell_index(&c->p, c->ox + i / r, j / r, k / r);
}

static uint64_t track_site(const orc_ms *c, int64_t i, int64_t j, int64_t k)
{
    const int64_t r = c->p.ratio;
    const int64_t X = (int64_t)c->ox * r + i, NX = (int64_t)c->p.ncx * r, NY = (int64_t)c->p.ncy * r;
    return (uint64_t)(X + NX * (j + NY * k));
}

/* Eq. 6 for the window cells of columns [cx0, cx1): the direction of the sum of the
 * cell's atomistic spins (0 for a non-magnetic cell or a zero sum). */
static void average_cells(orc_ms *c, int32_t cx0, int32_t cx1)
{
    const int r = c->p.ratio;
    const int64_t nxw = (int64_t)c->p.wx * r, nyw = (int64_t)c->p.ncy * r;
    for (int32_t cz = 0; cz < c->p.ncz; ++cz)
        for (int32_t cy = 0; cy < c->p.ncy; ++cy)
            for (int32_t cx = cx0; cx < cx1; ++cx) {
                int64_t q = cell_index(&c->p, cx, cy, cz);
                double s[3] = {0.0, 0.0, 0.0};
                if (c->grain[q] >= 0)
                    for (int dk = 0; dk < r; ++dk)
                        for (int dj = 0; dj < r; ++dj)
                            for (int di = 0; di < r; ++di) {
                                int64_t i = (int64_t)(cx - c->ox) * r + di, j = (int64_t)cy * r + dj,
                                        k = (int64_t)cz * r + dk;
                                const double *Si = c->S + 3 * (i + nxw * (j + nyw * k));
                                for (int d = 0; d < 3; ++d) s[d] += Si[d];
                            }
                double n = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
                for (int d = 0; d < 3; ++d) c->m[3 * q + d] = n > 0.0 ? s[d] / n : 0.0;
            }
}

static double cell_temperature(const orc_ms *c, int64_t q, double t)
{
    int64_t cx = q % c->p.ncx, cy = (q / c->p.ncx) % c->p.ncy;
    return orc_temperature(&c->p.drv, (cx + 0.5) * c->p.cell, (cy + 0.5) * c->p.cell, t);
}

/* Thermalise the window sites of cell columns [cx0, cx1) from the cells' m (event index
 * `event` in the Philox counter). */
static void thermalise(orc_ms *c, int32_t cx0, int32_t cx1, double t, uint64_t event)
{
    const int r = c->p.ratio;
    const int64_t nxw = (int64_t)c->p.wx * r, nyw = (int64_t)c->p.ncy * r, nzw = (int64_t)c->p.ncz * r;
    for (int64_t k = 0; k < nzw; ++k)
        for (int64_t j = 0; j < nyw; ++j)
            for (int64_t i = (int64_t)(cx0 - c->ox) * r; i < (int64_t)(cx1 - c->ox) * r; ++i) {
                int64_t q = site_cell(c, i, j, k);
                double *Si = c->S + 3 * (i + nxw * (j + nyw * k));
                const double *mq = c->m + 3 * q;
                if (c->grain[q] < 0 || (mq[0] == 0.0 && mq[1] == 0.0 && mq[2] == 0.0)) {
                    Si[0] = Si[1] = Si[2] = 0.0;
                    continue;
                }
                double B[3];
                orc_ms_field(&c->p, (q % c->p.ncx + 0.5) * c->p.cell, t, B);
                double Bm = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
                double mr = orc_me(c->p.T_C, cell_temperature(c, q, t), c->p.mu_s, Bm);
                orc_cone_sample(mq, orc_theta_max(mr), c->p.drv.seed, track_site(c, i, j, k), event, Si);
            }
}

/* Whether cell column cx is in the simulated region (every column without a region). */
static int in_region(const orc_ms *c, int64_t cx)
{
    const int32_t g = c->p.margin;
    return g < 0 || (cx >= (int64_t)c->ox - g && cx < (int64_t)c->ox + c->p.wx + g);
}

/* m_e(T(t), |B_app(t)|) of every magnetic cell into me_store. */
static void store_me(orc_ms *c, double t)
{
    const orc_ms_params *p = &c->p;
    for (int64_t q = 0; q < c->nc; ++q) {
        if (c->grain[q] < 0) continue;
        double B[3];
        orc_ms_field(p, (q % p->ncx + 0.5) * p->cell, t, B);
        c->me_store[q] = orc_me(p->T_C, cell_temperature(c, q, t), p->mu_s, sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
    }
}

/* Place the window at cell column ox and thermalise all of it from the cells.  A window that
 * is already placed first hands its sites back to its cells by Eq. 6, as the trailing column
 * does when the window moves (Sec. II), unless the cells have been replaced since. */
int orc_ms_set_window(orc_ms *c, int32_t ox)
{
    if (ox < 0 || ox + c->p.wx > c->p.ncx) return -1;
    if (c->live) average_cells(c, c->ox, c->ox + c->p.wx);
    c->live = 1;
    c->ox = ox;
    /* every cell's m_e at the placement: a cell that stays frozen keeps it */
    store_me(c, (double)c->step * c->p.drv.dt);
    thermalise(c, ox, ox + c->p.wx, (double)c->step * c->p.drv.dt, (uint64_t)c->events);
    c->events += 1;
    return 0;
}

/* Move the window forward by one cell column (step 4 of the header). */
static void shift_forward(orc_ms *c, double t)
{
    const int r = c->p.ratio;
    const int64_t nxw = (int64_t)c->p.wx * r, nyw = (int64_t)c->p.ncy * r, nzw = (int64_t)c->p.ncz * r;
    average_cells(c, c->ox, c->ox + 1);
    for (int64_t k = 0; k < nzw; ++k)
        for (int64_t j = 0; j < nyw; ++j)
            for (int64_t i = 0; i + r < nxw; ++i)
                for (int d = 0; d < 3; ++d)
                    c->S[3 * (i + nxw * (j + nyw * k)) + d] = c->S[3 * (i + r + nxw * (j + nyw * k)) + d];
    c->ox += 1;
    thermalise(c, c->ox + c->p.wx - 1, c->ox + c->p.wx, t, (uint64_t)c->events);
    c->events += 1;
}

/* ------------------------------------------------------------------------- */
/* Atomistic step of the window (stage 2) */

/* Exchange sum sum_j J S_j of site (i, j, k) over its same-grain bonds, with the window
 * spins V and, across the window's x faces, the micromagnetic cells m. */
static void site_exchange(const orc_ms *c, const double *V, int64_t i, int64_t j, int64_t k, int32_t g,
                          double ex[3])
{
    const int r = c->p.ratio;
    const int64_t nxw = (int64_t)c->p.wx * r, nyw = (int64_t)c->p.ncy * r, nzw = (int64_t)c->p.ncz * r;
    ex[0] = ex[1] = ex[2] = 0.0;
    const int64_t off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int b = 0; b < 6; ++b) {
        int64_t ii = i + off[b][0], jj = j + off[b][1], kk = k + off[b][2];
        if (jj < 0 || jj >= nyw || kk < 0 || kk >= nzw) continue;
        const double *v;
        int32_t gj;
        if (ii >= 0 && ii < nxw) {
            gj = c->grain[site_cell(c, ii, jj, kk)];
            v = V + 3 * (ii + nxw * (jj + nyw * kk));
        } else {
            int64_t cx = c->ox + (ii < 0 ? -1 : c->p.wx);
            if (cx < 0 || cx >= c->p.ncx) continue;
            int64_t q = cell_index(&c->p, cx, jj / r, kk / r);
            gj = c->grain[q];
            v = c->m + 3 * q;
        }
        if (gj != g) continue;
        for (int d = 0; d < 3; ++d) ex[d] += c->p.J * v[d];
    }
}

static void atom_rhs(const orc_ms *c, const double S[3], const double B[3], double f[3])
{
    orc_params q = c->p.drv;
    q.alpha = c->p.lambda;
    orc_llg_rhs(&q, S, B, f);
}

static int atom_step(orc_ms *c)
{
    const orc_ms_params *p = &c->p;
    const int r = p->ratio;
    const int64_t nxw = (int64_t)p->wx * r, nyw = (int64_t)p->ncy * r, nzw = (int64_t)p->ncz * r;
    const int64_t n = c->nw;
    const double dt = p->drv.dt, t = (double)c->step * dt, a = p->cell / r;
    double *Bth = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *f1 = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *Sp = (double *)calloc(3 * (size_t)n, sizeof(double));
    if (!Bth || !f1 || !Sp) { free(Bth); free(f1); free(Sp); return -1; }
    /* thermal field, field at S and predictor */
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        int64_t i = s % nxw, j = (s / nxw) % nyw, k = s / (nxw * nyw);
        int32_t g = c->grain[site_cell(c, i, j, k)];
        if (g < 0) continue;
        double T = orc_temperature(&p->drv, ((double)c->ox * r + i + 0.5) * a, (j + 0.5) * a, t);
        double sigma = sqrt(2.0 * p->lambda * ORC_KB * T / (p->drv.gamma * p->mu_s * dt));
        double xi[3];
        orc_thermal_normals(p->drv.seed, track_site(c, i, j, k), (uint64_t)c->step, xi);
        for (int d = 0; d < 3; ++d) Bth[3 * s + d] = sigma * xi[d];
        double ex[3], B[3], Bapp[3];
        orc_ms_field(p, ((double)c->ox * r + i + 0.5) * a, t, Bapp);
        site_exchange(c, c->S, i, j, k, g, ex);
        const double *Si = c->S + 3 * s;
        const double *bd = c->Bd + 3 * site_cell(c, i, j, k);
        B[0] = ex[0] / p->mu_s + Bapp[0] + Bth[3 * s] + bd[0];
        B[1] = ex[1] / p->mu_s + Bapp[1] + Bth[3 * s + 1] + bd[1];
        B[2] = ex[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Si[2] + Bapp[2] + Bth[3 * s + 2] + bd[2];
        atom_rhs(c, Si, B, f1 + 3 * s);
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = Si[d] + dt * f1[3 * s + d];
        double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d) Sp[3 * s + d] = v[d] / nv;
    }
    /* field at S' and corrector */
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        int64_t i = s % nxw, j = (s / nxw) % nyw, k = s / (nxw * nyw);
        int32_t g = c->grain[site_cell(c, i, j, k)];
        if (g < 0) continue;
        double ex[3], B[3], f2[3], Bapp[3];
        orc_ms_field(p, ((double)c->ox * r + i + 0.5) * a, t, Bapp);
        site_exchange(c, Sp, i, j, k, g, ex);
        const double *Spi = Sp + 3 * s;
        const double *bd = c->Bd + 3 * site_cell(c, i, j, k);
        B[0] = ex[0] / p->mu_s + Bapp[0] + Bth[3 * s] + bd[0];
        B[1] = ex[1] / p->mu_s + Bapp[1] + Bth[3 * s + 1] + bd[1];
        B[2] = ex[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Spi[2] + Bapp[2] + Bth[3 * s + 2] + bd[2];
        atom_rhs(c, Spi, B, f2);
        double *Si = c->S + 3 * s;
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = Si[d] + 0.5 * dt * (f1[3 * s + d] + f2[d]);
        double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d) Si[d] = v[d] / nv;
    }
    free(Bth); free(f1); free(Sp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Micromagnetic RK4 step (stage 3) */

/* dm/dt of cell q for the stage values V, with per-cell m_e and T at t_n. */
static void mm_rate(const orc_ms *c, const double *V, int64_t q, double me, double T, const double *Bapp,
                    double k[3])
{
    const orc_ms_params *p = &c->p;
    int64_t cx = q % p->ncx, cy = (q / p->ncx) % p->ncy, cz = q / ((int64_t)p->ncx * p->ncy);
    const int64_t off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    const double *mq = V + 3 * q;
    double lap[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 6; ++b) {
        int64_t x = cx + off[b][0], y = cy + off[b][1], z = cz + off[b][2];
        if (x < 0 || x >= p->ncx || y < 0 || y >= p->ncy || z < 0 || z >= p->ncz) continue;
        int64_t qn = cell_index(p, x, y, z);
        if (c->grain[qn] != c->grain[q]) continue;
        for (int d = 0; d < 3; ++d) lap[d] += (V[3 * qn + d] - mq[d]) / (p->cell * p->cell);
    }
    double cex = 2.0 * p->A0 * me * me / (p->Ms0 * me), cK = 2.0 * p->K0 * me * me * me / (p->Ms0 * me);
    if (!(me > 0.0)) cex = cK = 0.0;
    const double *bd = c->Bd + 3 * q;
    double B[3] = {cex * lap[0] + Bapp[0] + bd[0], cex * lap[1] + Bapp[1] + bd[1],
                   cex * lap[2] + cK * mq[2] + Bapp[2] + bd[2]};
    orc_params pp = p->drv;
    pp.alpha = orc_ms_alpha(p, T);
    orc_llg_rhs(&pp, mq, B, k);
}

static int mm_step(orc_ms *c)
{
    const orc_ms_params *p = &c->p;
    const int64_t nc = c->nc;
    const double dt = p->drv.dt, t = (double)c->step * dt;
    double *V = (double *)malloc(sizeof(double) * 3 * (size_t)nc);
    double *K = (double *)malloc(sizeof(double) * 3 * (size_t)nc);
    double *acc = (double *)calloc(3 * (size_t)nc, sizeof(double));
    double *me = (double *)malloc(sizeof(double) * (size_t)nc);
    double *T = (double *)malloc(sizeof(double) * (size_t)nc);
    if (!V || !K || !acc || !me || !T) { free(V); free(K); free(acc); free(me); free(T); return -1; }
    double *Bq = (double *)malloc(sizeof(double) * 3 * (size_t)nc);
    if (!Bq) { free(V); free(K); free(acc); free(me); free(T); return -1; }
    for (int64_t q = 0; q < nc; ++q) {
        orc_ms_field(p, (q % p->ncx + 0.5) * p->cell, t, Bq + 3 * q);
        double Bm = sqrt(Bq[3 * q] * Bq[3 * q] + Bq[3 * q + 1] * Bq[3 * q + 1] + Bq[3 * q + 2] * Bq[3 * q + 2]);
        T[q] = cell_temperature(c, q, t);
        me[q] = orc_me(p->T_C, T[q], p->mu_s, Bm);
    }
    /* the simulated region's cells keep this step's m_e; frozen cells keep theirs */
    for (int64_t q = 0; q < nc; ++q)
        if (c->grain[q] >= 0 && in_region(c, q % p->ncx)) c->me_store[q] = me[q];
#define ORC_EVOLVED(q) \
    (c->grain[q] >= 0 && ((q) % p->ncx < c->ox || (q) % p->ncx >= c->ox + p->wx) && in_region(c, (q) % p->ncx))
    memcpy(V, c->m, sizeof(double) * 3 * (size_t)nc);
    const double cstage[4] = {0.5, 0.5, 1.0, 0.0}, wstage[4] = {1.0, 2.0, 2.0, 1.0};
    for (int s = 0; s < 4; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < nc; ++q) {
            if (!ORC_EVOLVED(q)) continue;
            mm_rate(c, V, q, me[q], T[q], Bq + 3 * q, K + 3 * q);
        }
        for (int64_t q = 0; q < nc; ++q) {
            if (!ORC_EVOLVED(q)) continue;
            for (int d = 0; d < 3; ++d) {
                acc[3 * q + d] += wstage[s] * K[3 * q + d];
                V[3 * q + d] = c->m[3 * q + d] + cstage[s] * dt * K[3 * q + d];
            }
        }
    }
    for (int64_t q = 0; q < nc; ++q) {
        if (!ORC_EVOLVED(q)) continue;
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = c->m[3 * q + d] + dt / 6.0 * acc[3 * q + d];
        double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d) c->m[3 * q + d] = v[d] / nv;
    }
#undef ORC_EVOLVED
    free(V); free(K); free(acc); free(me); free(T); free(Bq);
    return 0;
}

void orc_demag_field(const orc_ms_params *p, const double *M, double *Bd);

/* Stage 1b (with demag): the cells' magnetisation at t_n -- window cells
 * M = (mu_s / V) sum_j m_j (Eq. 6), the others M = Ms0 m_e(T, |B_app|) m -- and
 * B_d = -mu0 N * M (Eq. 7) on every cell, frozen for the step. */
static int demag_stage(orc_ms *c)
{
    const orc_ms_params *p = &c->p;
    const int r = p->ratio;
    const int64_t nc = c->nc, nxw = (int64_t)p->wx * r, nyw = (int64_t)p->ncy * r;
    const double t = (double)c->step * p->drv.dt, V = p->cell * p->cell * p->cell;
    double *M = (double *)calloc(3 * (size_t)nc, sizeof(double));
    if (!M) return -1;
    for (int64_t q = 0; q < nc; ++q) {
        if (c->grain[q] < 0) continue;
        int64_t cx = q % p->ncx, cy = (q / p->ncx) % p->ncy, cz = q / ((int64_t)p->ncx * p->ncy);
        if (cx >= c->ox && cx < c->ox + p->wx) {
            for (int dk = 0; dk < r; ++dk)
                for (int dj = 0; dj < r; ++dj)
                    for (int di = 0; di < r; ++di) {
                        int64_t i = (cx - c->ox) * r + di, j = cy * r + dj, k = cz * r + dk;
                        const double *Si = c->S + 3 * (i + nxw * (j + nyw * k));
                        for (int d = 0; d < 3; ++d) M[3 * q + d] += p->mu_s / V * Si[d];
                    }
        } else {
            /* a frozen cell (outside the simulated region) keeps its stored m_e */
            double me = c->me_store[q];
            if (in_region(c, cx)) {
                double B[3];
                orc_ms_field(p, (cx + 0.5) * p->cell, t, B);
                me = orc_me(p->T_C, cell_temperature(c, q, t), p->mu_s, sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
            }
            for (int d = 0; d < 3; ++d) M[3 * q + d] = p->Ms0 * me * c->m[3 * q + d];
        }
    }
    orc_demag_field(p, M, c->Bd);
    free(M);
    return 0;
}

/* The window's target column: centred on the laser spot at time t, within the track. */
int32_t orc_ms_target(const orc_ms_params *p, double t)
{
    double xc = p->drv.x0 + p->drv.vx * t;
    double f = floor(xc / p->cell - 0.5 * p->wx + 0.5);
    if (f < 0.0) f = 0.0;
    if (f > (double)(p->ncx - p->wx)) f = (double)(p->ncx - p->wx);
    return (int32_t)f;
}

/* n_steps coupled steps (stages 1-4 of the header); follow != 0 moves the window with the
 * laser spot after each step.  Returns 0, or -1 on allocation failure. */
int orc_ms_run(orc_ms *c, int64_t n_steps, int32_t follow)
{
    for (int64_t s = 0; s < n_steps; ++s) {
        average_cells(c, c->ox, c->ox + c->p.wx);
        if (c->p.demag && demag_stage(c) != 0) return -1;
        if (atom_step(c) != 0) return -1;
        if (mm_step(c) != 0) return -1;
        c->step += 1;
        if (follow) {
            double t = (double)c->step * c->p.drv.dt;
            int32_t target = orc_ms_target(&c->p, t);
            while (c->ox < target) shift_forward(c, t);
        }
    }
    /* the window cells report the Eq. 6 directions of the current spins */
    average_cells(c, c->ox, c->ox + c->p.wx);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Read-back of the written track: a stand-in for the read head (Sec. III), whose
 * tunnel-junction model is not part of the paper.  Bit b covers the cells whose centre x lies
 * in [x_start + b L, x_start + (b + 1) L) and whose row cy lies in [cy0, cy1), all layers; its
 * signal is the mean m_z over the magnetic cells there (0 when there are none), and it reads
 * as 1 when the signal is negative (a '1' is written along -z). */
void orc_ms_read_track(const orc_ms *c, double x_start, double bit_len, int32_t n_bits, int32_t cy0, int32_t cy1,
                       double *signal, uint8_t *bits)
{
    for (int32_t b = 0; b < n_bits; ++b) {
        double sum = 0.0;
        int64_t count = 0;
        for (int32_t cz = 0; cz < c->p.ncz; ++cz)
            for (int32_t cy = cy0; cy < cy1; ++cy)
                for (int32_t cx = 0; cx < c->p.ncx; ++cx) {
                    double x = (cx + 0.5) * c->p.cell;
                    if (!(x >= x_start + b * bit_len && x < x_start + (b + 1) * bit_len)) continue;
                    int64_t q = cell_index(&c->p, cx, cy, cz);
                    if (c->grain[q] < 0) continue;
                    sum += c->m[3 * q + 2];
                    count += 1;
                }
        signal[b] = count > 0 ? sum / (double)count : 0.0;
        if (bits) bits[b] = signal[b] < 0.0 ? 1 : 0;
    }
}

/* ------------------------------------------------------------------------- */
/* Demagnetising field (Eq. 7): H = -N * M, a convolution of the cells' magnetisation with
 * the demagnetising tensor of uniformly magnetised cuboid cells (Newell, Williams and
 * Dunlop, J. Geophys. Res. 98, 9551 (1993)).  The tensor between two cells at offset
 * (X, Y, Z) is the second difference over the cell edges of the functions f (diagonal) and
 * g (off-diagonal) below, divided by 4 pi dx dy dz; beyond ORC_DIPOLE_CELLS cell edges it is
 * the point-dipole tensor -(V / 4 pi r^3)(3 r r / r^2 - I), where the second difference
 * cancels to rounding.  Atomistic moments enter through Eq. 6, M = (mu_s / V) sum_j m_j;
 * micromagnetic cells carry M = Ms0 m_e(T) m. */
#define ORC_DIPOLE_CELLS 40.0

static double asinh_ratio(double a, double b)   /* asinh(a / b), 0 when b = 0 */
{
    return b > 0.0 ? asinh(a / b) : 0.0;
}

static double atan_ratio(double a, double b)    /* atan(a / b), 0 when b = 0 */
{
    return b != 0.0 ? atan(a / b) : 0.0;
}

double orc_newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    r += 0.5 * y * (z2 - x2) * asinh_ratio(y, sqrt(x2 + z2));
    r += 0.5 * z * (y2 - x2) * asinh_ratio(z, sqrt(x2 + y2));
    r -= x * y * z * atan_ratio(y * z, x * R);
    r += (2.0 * x2 - y2 - z2) * R / 6.0;
    return r;
}

double orc_newell_g(double x, double y, double z)
{
    double sx = x < 0 ? -1.0 : 1.0, sy = y < 0 ? -1.0 : 1.0;   /* g is odd in x and y, even in z */
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    r += x * y * z * asinh_ratio(z, sqrt(x2 + y2));
    r += y * (3.0 * z2 - y2) * asinh_ratio(x, sqrt(y2 + z2)) / 6.0;
    r += x * (3.0 * z2 - x2) * asinh_ratio(y, sqrt(x2 + z2)) / 6.0;
    r -= z2 * z * atan_ratio(x * y, z * R) / 6.0;
    r -= 0.5 * z * y2 * atan_ratio(x * z, y * R);
    r -= 0.5 * z * x2 * atan_ratio(y * z, x * R);
    r -= x * y * R / 3.0;
    return sx * sy * r;
}

/* second difference sum_{i,j,k} c_i c_j c_k F(X + i dx, Y + j dy, Z + k dz), c_0 = 2, c_+-1 = -1 */
static double second_difference(double (*F)(double, double, double), double X, double Y, double Z, double dx,
                                double dy, double dz)
{
    static const double c[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j)
            for (int k = -1; k <= 1; ++k)
                s += c[i + 1] * c[j + 1] * c[k + 1] * F(X + i * dx, Y + j * dy, Z + k * dz);
    return s;
}

static double f_yxz(double x, double y, double z) { return orc_newell_f(y, x, z); }
static double f_zyx(double x, double y, double z) { return orc_newell_f(z, y, x); }
static double g_xzy(double x, double y, double z) { return orc_newell_g(x, z, y); }
static double g_yzx(double x, double y, double z) { return orc_newell_g(y, z, x); }

/* The six components (xx, yy, zz, xy, xz, yz) of the tensor between cells at offset (X, Y, Z)
 * for cells of edges (dx, dy, dz). */
void orc_demag_tensor(double X, double Y, double Z, double dx, double dy, double dz, double N[6])
{
    double r = sqrt(X * X + Y * Y + Z * Z);
    double lmax = fmax(dx, fmax(dy, dz));
    if (r > ORC_DIPOLE_CELLS * lmax) {
        double V = dx * dy * dz, pre = -V / (4.0 * ORC_PI * r * r * r), r2 = r * r;
        N[0] = pre * (3.0 * X * X / r2 - 1.0);
        N[1] = pre * (3.0 * Y * Y / r2 - 1.0);
        N[2] = pre * (3.0 * Z * Z / r2 - 1.0);
        N[3] = pre * 3.0 * X * Y / r2;
        N[4] = pre * 3.0 * X * Z / r2;
        N[5] = pre * 3.0 * Y * Z / r2;
        return;
    }
    double k = 1.0 / (4.0 * ORC_PI * dx * dy * dz);
    N[0] = k * second_difference(orc_newell_f, X, Y, Z, dx, dy, dz);
    N[1] = k * second_difference(f_yxz, X, Y, Z, dx, dy, dz);
    N[2] = k * second_difference(f_zyx, X, Y, Z, dx, dy, dz);
    N[3] = k * second_difference(orc_newell_g, X, Y, Z, dx, dy, dz);
    N[4] = k * second_difference(g_xzy, X, Y, Z, dx, dy, dz);
    N[5] = k * second_difference(g_yzx, X, Y, Z, dx, dy, dz);
}

/* B_d = mu0 H_d = -mu0 sum_j N(r_i - r_j) M_j [T] on every cell, by direct summation, for the
 * cell magnetisations M [A/m] (AoS 3 nc). */
void orc_demag_field(const orc_ms_params *p, const double *M, double *Bd)
{
    const double mu0 = 1.25663706212e-6;
    const int64_t nc = (int64_t)p->ncx * p->ncy * p->ncz;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < nc; ++i) {
        int64_t ix = i % p->ncx, iy = (i / p->ncx) % p->ncy, iz = i / ((int64_t)p->ncx * p->ncy);
        double h[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < nc; ++j) {
            const double *Mj = M + 3 * j;
            if (Mj[0] == 0.0 && Mj[1] == 0.0 && Mj[2] == 0.0) continue;
            int64_t jx = j % p->ncx, jy = (j / p->ncx) % p->ncy, jz = j / ((int64_t)p->ncx * p->ncy);
            double N[6];
            orc_demag_tensor((ix - jx) * p->cell, (iy - jy) * p->cell, (iz - jz) * p->cell, p->cell, p->cell, p->cell,
                             N);
            h[0] += N[0] * Mj[0] + N[3] * Mj[1] + N[4] * Mj[2];
            h[1] += N[3] * Mj[0] + N[1] * Mj[1] + N[5] * Mj[2];
            h[2] += N[4] * Mj[0] + N[5] * Mj[1] + N[2] * Mj[2];
        }
        for (int d = 0; d < 3; ++d) Bd[3 * i + d] = -mu0 * h[d];
    }
}
