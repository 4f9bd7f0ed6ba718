/*
 * cx_oracle.c -- plain FP64 CPU oracle for the bacteria/nutrient
 * chemotaxis system of Leyva, Malaga & Plaza, "The effects of nutrient
 * chemotaxis on bacterial aggregation patterns with non-linear degenerate
 * cross diffusion" (Sec. 2.4, Eq. ka-chem-model, and its general form
 * Eq. ka-model-dim with the kinetics of Eq. goodkinetics).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library
 * against; it is slow on purpose and is never called by the product path.
 * Only tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant with the
 * CUDA sources.
 *
 * Everything is written in the order the definitions give it, in FP64,
 * one cell (or one face) at a time.  Build with -ffp-contract=off so that
 * no multiply-add is fused and the result is the same on x86-64 and arm64.
 * Built a second time with -fopenmp, the loops over rows of the right-hand
 * side and over cells of the updates run on several host threads; each
 * cell's arithmetic and its order are the same, so both builds give the
 * same bits (only the baseline timing uses the threaded build).
 *
 * Discrete problem (the paper states the PDE and "explicit Runge-Kutta +
 * finite differences" only, Sec. 3; the readings below are the ones this
 * project fixes):
 *   - cell-centred nx*ny grid of spacing dx; cell (i,j) has its centre at
 *     x = (i + 1/2 - nx/2) dx, y = (j + 1/2 - ny/2) dx, row-major j*nx + i;
 *   - on each face between a lower/left cell L and an upper/right cell R:
 *       s_f = (s_L+s_R)/2, n_f = (n_L+n_R)/2, b_f = (b_L+b_R)/2,
 *       diffusive flux    Fd = s_f n_f b_f (b_R-b_L)/dx            (Eq. CoefCrsDif)
 *       chemotactic flux  Fc = chi(n_f) s_f n_f m_f (n_R-n_L)/dx   (Eq. chemflux)
 *         chi(n) = chi0/(1+n)^2 (receptor law, Eq. receptor_law, normalised)
 *                or chi0      (constant law, Sec. 4.1, Eq. velo-system)
 *         m_f = b_f^2 (central) or b_donor^2, donor = the lower-n side
 *       nutrient flux     G  = Dn (n_R-n_L)/dx
 *     faces on the domain boundary carry zero flux (Eq. bconds);
 *   - per cell: rb = (PhiE-PhiW + PhiN-PhiS)/dx + theta n b,   Phi = Fd - Fc
 *               rn = (GE-GW + GN-GS)/dx - n b                  (kappa = 1)
 *   - forward Euler: u' = u + dt r(u);
 *     Heun (second-order Runge-Kutta, Sec. 3): u' = u + dt/2 (r(u) + r(u + dt r(u)));
 *   - sigma = sigma0 (1 + a Delta) (Eq. CoefCrsDif), Delta drawn per cell
 *     from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), uniform on
 *     [-1,1) or triangular on (-1,1) (Sec. 3), either once or per step.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from the definition in Salmon et al. (SC'11):
 * one round maps (c0,c1,c2,c3) with multipliers M0, M1 to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
 * and the key is bumped by the Weyl constants between rounds.        */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The random perturbation Delta of cell `idx` at time step `step`
 * (Sec. 3: "on every grid point and at each time step", triangular on
 * [-1,1]).  Counter = (idx lo, idx hi, step lo, step hi), key = seed.
 * Two 53-bit integers k_a, k_b are formed from the four output words;
 * U_a = k_a 2^-53 is uniform on [0,1).
 *   dist 0 (uniform on [-1,1)):  Delta = 2 U_a - 1
 *   dist 1 (triangular):         Delta = U_a + U_b - 1
 * Both are evaluated exactly in integers and scaled by 2^-53 (exact). */
double orc_noise_delta(uint64_t seed, uint64_t idx, uint64_t step, int dist)
{
    uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32),
                       (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int64_t ka = (int64_t)(((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11));
    int64_t kb = (int64_t)(((uint64_t)w[2] << 21) | (uint64_t)(w[3] >> 11));
    int64_t two53 = (int64_t)1 << 53;
    int64_t num = (dist == 0) ? (2 * ka - two53) : (ka + kb - two53);
    return ldexp((double)num, -53);
}

/* FP32 recipe, used when the state is held in FP32 and sigma is redrawn
 * every step: one Philox block serves four consecutive cells, block counter
 * (q lo, q hi, step lo, step hi) with q = idx >> 2, and cell idx takes word
 * w[h], h = idx & 3, as two 16-bit integers j_a = w[h] >> 16 and
 * j_b = w[h] & 0xffff:
 *   dist 0:  Delta = (2 j_a - 2^16) 2^-16,   dist 1:  Delta = (j_a + j_b - 2^16) 2^-16,
 * exact in float, then sigma = sigma0 (1 + a Delta) with each float
 * operation rounded on its own. */
float orc_noise_sigma_f32(uint64_t seed, uint64_t idx, uint64_t step, int dist,
                          float sigma0, float amp)
{
    uint64_t q = idx >> 2;
    int h = (int)(idx & 3);
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32),
                       (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int32_t ja = (int32_t)(w[h] >> 16), jb = (int32_t)(w[h] & 0xffffu);
    int32_t num = (dist == 0) ? (2 * ja - (1 << 16)) : (ja + jb - (1 << 16));
    float d = (float)num * 0x1p-16f;
    float t = amp * d;
    float s = 1.0f + t;
    return sigma0 * s;
}

void orc_sigma_field_f32(int nx, int ny, uint64_t seed, uint64_t step, double sigma0,
                         double amp, int dist, double *sigma)
{
    float s0 = (float)sigma0, a = (float)amp;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            uint64_t idx = (uint64_t)j * (uint64_t)nx + (uint64_t)i;
            sigma[idx] = (double)orc_noise_sigma_f32(seed, idx, step, dist, s0, a);
        }
}

/* sigma_ij = sigma0 (1 + a Delta_ij)   (Eq. CoefCrsDif) */
void orc_sigma_field(int nx, int ny, uint64_t seed, uint64_t step,
                     double sigma0, double amp, int dist, double *sigma)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            uint64_t idx = (uint64_t)j * (uint64_t)nx + (uint64_t)i;
            double d = orc_noise_delta(seed, idx, step, dist);
            double t = amp * d;
            double s = 1.0 + t;
            sigma[idx] = sigma0 * s;
        }
}

/* Initial state (Eq. inicond, Eq. inibacexp): n = n0 everywhere and a
 * Gaussian inoculum b = bM exp(-r^2 / r0sq) centred on the domain, read as
 * cut to zero where r^2 / r0sq > 40 (a real inoculum has compact support;
 * the cut changes its mass by less than e^-40 and keeps every nonzero value
 * a normal FP32 number, so an FP32 and an FP64 state start alike instead of
 * differing wherever FP32 underflows). */
void orc_initial_state(int nx, int ny, double dx, double n0, double bM,
                       double r0sq, double *b, double *n)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = ((double)i + 0.5 - 0.5 * (double)nx) * dx;
            double y = ((double)j + 0.5 - 0.5 * (double)ny) * dx;
            double r2 = x * x + y * y;
            size_t p = (size_t)j * (size_t)nx + (size_t)i;
            double q = -r2 / r0sq;
            b[p] = q < -40.0 ? 0.0 : bM * exp(q);
            n[p] = n0;
        }
}

/* ------------------------------------------------------------------ */
/* Face fluxes between a lower/left cell L and an upper/right cell R.  */
typedef struct {
    double dx, Dn, theta, chi0;
    int chemo_law; /* 0 receptor chi0/(1+n)^2, 1 constant chi0 */
    int mobility;  /* 0 central b_f^2, 1 donor-cell b^2 */
} orc_coeffs;

static void face_flux(const orc_coeffs *c, double sL, double sR, double nL,
                      double nR, double bL, double bR, double *phi, double *g)
{
    double sf = 0.5 * (sL + sR);
    double nf = 0.5 * (nL + nR);
    double bf = 0.5 * (bL + bR);
    /* sigma n b grad b */
    double Fd = sf * nf * bf * (bR - bL) / c->dx;
    /* chemotactic sensitivity at the face */
    double chi;
    if (c->chemo_law == 0)
        chi = c->chi0 / ((1.0 + nf) * (1.0 + nf));
    else
        chi = c->chi0;
    /* b^2 at the face */
    double m;
    if (c->mobility == 0)
        m = bf * bf;
    else
        m = (nR >= nL) ? bL * bL : bR * bR;
    /* sigma n b^2 chi(n) grad n */
    double Fc = chi * sf * nf * m * (nR - nL) / c->dx;
    *phi = Fd - Fc;
    *g = c->Dn * (nR - nL) / c->dx;
}

/* Right-hand side r(u) of the semi-discrete system for every cell. */
static void rhs(int nx, int ny, const orc_coeffs *c, const double *sigma,
                const double *b, const double *n, double *rb, double *rn)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t P = (size_t)j * (size_t)nx + (size_t)i;
            double phiW = 0.0, phiE = 0.0, phiS = 0.0, phiN = 0.0;
            double gW = 0.0, gE = 0.0, gS = 0.0, gN = 0.0;
            if (i > 0) {
                size_t Q = P - 1;
                face_flux(c, sigma[Q], sigma[P], n[Q], n[P], b[Q], b[P], &phiW, &gW);
            }
            if (i < nx - 1) {
                size_t Q = P + 1;
                face_flux(c, sigma[P], sigma[Q], n[P], n[Q], b[P], b[Q], &phiE, &gE);
            }
            if (j > 0) {
                size_t Q = P - (size_t)nx;
                face_flux(c, sigma[Q], sigma[P], n[Q], n[P], b[Q], b[P], &phiS, &gS);
            }
            if (j < ny - 1) {
                size_t Q = P + (size_t)nx;
                face_flux(c, sigma[P], sigma[Q], n[P], n[Q], b[P], b[Q], &phiN, &gN);
            }
            double divb = ((phiE - phiW) + (phiN - phiS)) / c->dx;
            double divn = ((gE - gW) + (gN - gS)) / c->dx;
            double r = n[P] * b[P];
            rb[P] = divb + c->theta * r;
            rn[P] = divn - r;
        }
}

void orc_rhs(int nx, int ny, double dx, double Dn, double theta, double chi0,
             int chemo_law, int mobility, const double *sigma, const double *b,
             const double *n, double *rb, double *rn)
{
    orc_coeffs c = {dx, Dn, theta, chi0, chemo_law, mobility};
    rhs(nx, ny, &c, sigma, b, n, rb, rn);
}

/* One forward-Euler step: u' = u + dt r(u). */
int orc_step_euler(int nx, int ny, double dx, double dt, double Dn,
                   double theta, double chi0, int chemo_law, int mobility,
                   const double *sigma, const double *b, const double *n,
                   double *b_out, double *n_out)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *rb = (double *)malloc(N * sizeof(double));
    double *rn = (double *)malloc(N * sizeof(double));
    if (!rb || !rn) { free(rb); free(rn); return -1; }
    orc_coeffs c = {dx, Dn, theta, chi0, chemo_law, mobility};
    rhs(nx, ny, &c, sigma, b, n, rb, rn);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < N; ++p) {
        b_out[p] = b[p] + dt * rb[p];
        n_out[p] = n[p] + dt * rn[p];
    }
    free(rb); free(rn);
    return 0;
}

/* One Heun step (second-order Runge-Kutta):
 *   u* = u + dt r(u);  u' = u + (dt/2) (r(u) + r(u*)).  sigma is the same
 * field in both stages (it is redrawn per time step, not per stage). */
int orc_step_heun(int nx, int ny, double dx, double dt, double Dn,
                  double theta, double chi0, int chemo_law, int mobility,
                  const double *sigma, const double *b, const double *n,
                  double *b_out, double *n_out)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *rb1 = (double *)malloc(N * sizeof(double));
    double *rn1 = (double *)malloc(N * sizeof(double));
    double *rb2 = (double *)malloc(N * sizeof(double));
    double *rn2 = (double *)malloc(N * sizeof(double));
    double *bs = (double *)malloc(N * sizeof(double));
    double *ns = (double *)malloc(N * sizeof(double));
    int ok = rb1 && rn1 && rb2 && rn2 && bs && ns;
    if (ok) {
        orc_coeffs c = {dx, Dn, theta, chi0, chemo_law, mobility};
        rhs(nx, ny, &c, sigma, b, n, rb1, rn1);
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < N; ++p) {
            bs[p] = b[p] + dt * rb1[p];
            ns[p] = n[p] + dt * rn1[p];
        }
        rhs(nx, ny, &c, sigma, bs, ns, rb2, rn2);
        double h = 0.5 * dt;
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < N; ++p) {
            b_out[p] = b[p] + h * (rb1[p] + rb2[p]);
            n_out[p] = n[p] + h * (rn1[p] + rn2[p]);
        }
    }
    free(rb1); free(rn1); free(rb2); free(rn2); free(bs); free(ns);
    return ok ? 0 : -1;
}

/* Run `nsteps` steps in place starting at time-step index `step0`.
 * scheme 0 Euler, 1 Heun.  noise_mode 0: `sigma` is a fixed field and is
 * used as given; noise_mode 1: sigma is redrawn before every step m from
 * (seed, cell, m) with sigma0, amp, dist and written into `sigma`, by the
 * FP64 recipe (recipe 0) or the FP32 recipe (recipe 1). */
int orc_run(int nx, int ny, double dx, double dt, double Dn, double theta,
            double chi0, int chemo_law, int mobility, int scheme,
            int noise_mode, int recipe, uint64_t seed, double sigma0, double amp, int dist,
            int64_t step0, int64_t nsteps, double *sigma, double *b, double *n)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *b2 = (double *)malloc(N * sizeof(double));
    double *n2 = (double *)malloc(N * sizeof(double));
    if (!b2 || !n2) { free(b2); free(n2); return -1; }
    int rc = 0;
    for (int64_t m = 0; m < nsteps && rc == 0; ++m) {
        if (noise_mode == 1 && recipe == 0)
            orc_sigma_field(nx, ny, seed, (uint64_t)(step0 + m), sigma0, amp, dist, sigma);
        else if (noise_mode == 1)
            orc_sigma_field_f32(nx, ny, seed, (uint64_t)(step0 + m), sigma0, amp, dist, sigma);
        if (scheme == 0)
            rc = orc_step_euler(nx, ny, dx, dt, Dn, theta, chi0, chemo_law, mobility,
                                sigma, b, n, b2, n2);
        else
            rc = orc_step_heun(nx, ny, dx, dt, Dn, theta, chi0, chemo_law, mobility,
                               sigma, b, n, b2, n2);
        memcpy(b, b2, N * sizeof(double));
        memcpy(n, n2, N * sizeof(double));
    }
    free(b2); free(n2);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics.  Sums use pairwise (recursive halving) summation over the
 * row-major cell order, so their rounding error stays O(log N). */
static double pairwise_sum(const double *x, size_t len)
{
    if (len <= 8) {
        double s = 0.0;
        for (size_t k = 0; k < len; ++k) s += x[k];
        return s;
    }
    size_t h = len / 2;
    return pairwise_sum(x, h) + pairwise_sum(x + h, len - h);
}

/* out[0] mass_b = dx^2 sum b
 * out[1] mass_n = dx^2 sum n
 * out[2] invariant = dx^2 sum (b + theta n)  (conserved by Eq. ka-model-dim
 *        with no-flux boundaries: the reaction terms cancel, the fluxes
 *        telescope)
 * out[3] min b, out[4] min n, out[5] max b
 * out[6] r_env = largest centre distance of a cell with b >= b_th (0 if none)
 * out[7] 1 if every b and n is finite, else 0
 * out[8] area_env = dx^2 x the number of cells with b >= b_th (the colony's
 *        area; sqrt(area_env / pi) is its equivalent radius) */
int orc_diagnostics(int nx, int ny, double dx, double theta, double b_th,
                    const double *b, const double *n, double out[9])
{
    size_t N = (size_t)nx * (size_t)ny;
    double *tmp = (double *)malloc(N * sizeof(double));
    if (!tmp) return -1;
    double area = dx * dx;
    out[0] = area * pairwise_sum(b, N);
    out[1] = area * pairwise_sum(n, N);
    for (size_t p = 0; p < N; ++p) tmp[p] = b[p] + theta * n[p];
    out[2] = area * pairwise_sum(tmp, N);
    free(tmp);
    double mnb = b[0], mnn = n[0], mxb = b[0], r2max = -1.0;
    long long above = 0;
    int finite = 1;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = (size_t)j * (size_t)nx + (size_t)i;
            if (!isfinite(b[p]) || !isfinite(n[p])) finite = 0;
            if (b[p] < mnb) mnb = b[p];
            if (n[p] < mnn) mnn = n[p];
            if (b[p] > mxb) mxb = b[p];
            if (b[p] >= b_th) {
                ++above;
                double x = ((double)i + 0.5 - 0.5 * (double)nx) * dx;
                double y = ((double)j + 0.5 - 0.5 * (double)ny) * dx;
                double r2 = x * x + y * y;
                if (r2 > r2max) r2max = r2;
            }
        }
    out[3] = mnb; out[4] = mnn; out[5] = mxb;
    out[6] = r2max >= 0.0 ? sqrt(r2max) : 0.0;
    out[7] = finite ? 1.0 : 0.0;
    out[8] = area * (double)above;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Explicit stability limit (the paper only says its time steps "showed
 * to be stable", Sec. 3).  Reading fixed by this project:
 *   B     = bM + theta n0   (upper estimate of b from local conservation
 *                            of b + theta n, Eq. mass-conser)
 *   Dmax  = max(Dn, sigma_max n0 B (1 + chi0 B))   (effective diffusivity,
 *                            Eq. D-tilde, evaluated at its largest factors)
 *   limit = min(dx^2 / (4 Dmax), 1 / (4 Dn / dx^2 + B)),
 * the second term keeping n >= 0 under forward Euler. */
double orc_dt_limit(double dx, double Dn, double theta, double chi0, double n0,
                    double bM, double sigma0, double amp)
{
    double B = bM + theta * n0;
    double sigma_max = sigma0 * (1.0 + fabs(amp));
    double Dchem = sigma_max * n0 * B * (1.0 + chi0 * B);
    double Dmax = Dn > Dchem ? Dn : Dchem;
    double l1 = dx * dx / (4.0 * Dmax);
    double l2 = 1.0 / (4.0 * Dn / (dx * dx) + B);
    return l1 < l2 ? l1 : l2;
}

/* ------------------------------------------------------------------ */
/* Host threads of the threaded build (1 in the plain build). */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
void orc_set_threads(int t) { if (t > 0) omp_set_num_threads(t); }
#else
int orc_threads(void) { return 1; }
void orc_set_threads(int t) { (void)t; }
#endif
