/*
 * prs_oracle.c -- plain, slow, FP64 CPU oracle for the Press-Ryden-Spergel (PRS)
 * domain-wall method of Correia & Martins, arXiv:1710.10420.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The product library shares
 * no code, header or constant with it and never calls it.
 *
 * Everything is written in the order and notation of the paper (Sec. II):
 *   Eq. 2  equation of motion   phi'' + alpha (dln a/dln eta) phi'/eta - lap phi = -a^beta dV/dphi
 *   Eq. 3  discrete Laplacian   (nearest-neighbour second difference, periodic)
 *   Eq. 4  velocity (kick)      dphi^{n+1/2} = [(1-delta) dphi^{n-1/2} + deta (lap phi^n - dV/dphi^n)]/(1+delta)
 *   Eq. 5  field (drift)        phi^{n+1} = phi^n + deta dphi^{n+1/2}
 *   Eq. 6  damping              delta = (1/2) alpha (deta/eta) (dln a/dln eta)
 *   Eq. 7  area per volume      A/V = dA sum_links delta_pm |grad phi| / (|phi,x|+|phi,y|+|phi,z|) / V
 *   Eq. 8  velocity             (gamma v)^2 = (1/2N) sum_walls E_k / V(phi)
 * with V(phi) = V0 (phi^2/phi0^2 - 1)^2 from the Lagrangian (Eq. 1).
 *
 * Readings taken where the paper is silent or garbled (each one is pinned by a
 * CPU test):
 *   - Eq. 2 prints "alpha^beta"; the force prefactor is the scale factor a^beta,
 *     with a(eta) = eta^m, m = dln a/dln eta (a = 1 at eta = 1).  PRS: beta = 0.
 *   - Eq. 3 is written for dx = 1; the Laplacian here carries 1/dx^2.
 *   - delta of step n uses eta_n = eta0 + n*deta, the time of phi^n (Eq. 6).
 *   - the first kick starts from dphi^{-1/2} = the initial velocity (no half kick).
 *   - V0 = pi^2 / (2 W0^2): a static kink is phi0 tanh(pi x / W0) for phi0 = 1;
 *     W0 = +inf gives V0 = 0 (free field).
 *   - Eq. 7 numerator is |grad phi| at the link midpoint: along the link the
 *     one-sided difference, across it the centred difference averaged over the
 *     two link ends.  A link crosses a wall iff (phi_s < 0) != (phi_t < 0).
 *     dA = dx^(D-1), V = (number of sites) dx^D.
 *   - Eq. 8: E_k is dphi^2 (so a boosted kink gives exactly (gamma u)^2); the
 *     walls are the sites with at least one of their 2D nearest neighbours of the
 *     opposite sign, each counted once; dphi is the stored dphi^{n-1/2}.  Wall
 *     sites with V(phi) = 0 are left out of the sum and of N, and counted.
 *   - Initial conditions: phi_s from SplitMix64 (Steele, Lea & Flood 2014) at
 *     counter idx+1 after the seed, top 24 bits k, phi = (2k+1) 2^-24 - 1.
 *
 * The adjoint (reverse-time derivative of the leapfrog step) and the two smooth
 * observables are not in the paper; they are the transpose of Eqs. 3-5 written
 * out by hand:
 *   forward  v' = c1 v + c2 (L phi - f(phi)),  phi' = phi + deta v'
 *   reverse  lt = lv' + deta lphi',  lphi = lphi' + c2 (L lt - f'(phi) lt),
 *            lv = c1 lt,  dJ/dalpha += sum lt (dc1/dalpha v + dc2/dalpha (L phi - f))
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add anywhere, no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t dims;      /* 2 or 3 */
    int32_t pad_;
    int64_t nx, ny, nz; /* box sides; nz = 1 for dims == 2 */
    double dx, deta, eta0;
    double alpha, beta, era_m; /* era_m = dln a / dln eta */
    double W0, phi0;
} orc_params;

typedef struct {
    double area_per_volume; /* Eq. 7 */
    double gamma_v;         /* sqrt of Eq. 8 */
    double sum_w;           /* sum over crossing links of the Eq. 7 weight */
    double sum_ratio;       /* sum over wall sites of dphi^2 / V(phi) */
    int64_t n_links;        /* links whose ends have opposite signs */
    int64_t n_wall;         /* wall sites */
    int64_t n_vzero;        /* wall sites with V(phi) == 0, excluded from Eq. 8 */
    int64_t n_nonfinite;    /* sites where phi or dphi is not finite */
} orc_diag;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ lattice */

static int64_t orc_sites(const orc_params* p) { return p->nx * p->ny * (p->dims == 3 ? p->nz : 1); }

static int64_t wrap(int64_t i, int64_t n) { return ((i % n) + n) % n; }

/* Linear index of (x, y, z) with periodic wrap; x runs fastest. */
static int64_t at(const orc_params* p, int64_t x, int64_t y, int64_t z)
{
    int64_t nz = p->dims == 3 ? p->nz : 1;
    return wrap(x, p->nx) + p->nx * (wrap(y, p->ny) + p->ny * wrap(z, nz));
}

static void coords(const orc_params* p, int64_t s, int64_t c[3])
{
    c[0] = s % p->nx;
    c[1] = (s / p->nx) % p->ny;
    c[2] = s / (p->nx * p->ny);
}

/* Site reached from s by moving `step` (+1 or -1) along axis d. */
static int64_t neighbour(const orc_params* p, int64_t s, int d, int step)
{
    int64_t c[3];
    coords(p, s, c);
    c[d] += step;
    return at(p, c[0], c[1], c[2]);
}

/* ---------------------------------------------------------- random numbers */

/* SplitMix64 output number idx (0-based) of the generator whose state starts at
 * `seed`: the state is advanced idx+1 times by the golden-ratio increment, then
 * passed through the published finaliser. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t idx)
{
    uint64_t z = seed + (idx + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform value in (-1, 1) from the top 24 bits; exactly representable in FP32. */
double orc_uniform(uint64_t seed, uint64_t idx)
{
    uint64_t k = orc_splitmix64(seed, idx) >> 40;
    return (double)(2u * k + 1u) * (1.0 / 16777216.0) - 1.0;
}

/* Random initial conditions: phi i.i.d. in (-1, 1), zero velocity. */
void orc_init_random(const orc_params* p, uint64_t seed, double* phi, double* v)
{
    int64_t S = orc_sites(p);
    for (int64_t s = 0; s < S; ++s) {
        phi[s] = orc_uniform(seed, (uint64_t)s);
        v[s] = 0.0;
    }
}

/* ------------------------------------------------------------ coefficients */

double orc_V0(const orc_params* p) { return ORC_PI * ORC_PI / (2.0 * p->W0 * p->W0); }

/* Coefficients of leapfrog step n (phi^n -> phi^{n+1}):
 * out[0] = c1 = (1-delta)/(1+delta), out[1] = c2 = deta/(1+delta),
 * out[2] = cV = 4 V0 a^beta / phi0^2 (the prefactor of phi (phi^2/phi0^2 - 1) in
 * a^beta dV/dphi), out[3] = delta, out[4] = d delta / d alpha. */
void orc_coeffs(const orc_params* p, int64_t n, double out[5])
{
    double eta = p->eta0 + (double)n * p->deta;              /* computed, not accumulated */
    double delta = 0.5 * p->alpha * p->deta * p->era_m / eta; /* Eq. 6 */
    double a_beta = 1.0;
    if (p->beta != 0.0) a_beta = pow(pow(eta, p->era_m), p->beta);
    out[0] = (1.0 - delta) / (1.0 + delta);
    out[1] = p->deta / (1.0 + delta);
    out[2] = 4.0 * orc_V0(p) * a_beta / (p->phi0 * p->phi0);
    out[3] = delta;
    out[4] = 0.5 * p->deta * p->era_m / eta;
}

/* ------------------------------------------------------------------ stepping */

/* Eq. 3 with 1/dx^2: sum over axes of the neighbour pair, minus 2D phi_s. */
static double laplacian(const orc_params* p, const double* f, int64_t s)
{
    double s2 = 0.0;
    for (int d = 0; d < p->dims; ++d) {
        double pair = f[neighbour(p, s, d, +1)] + f[neighbour(p, s, d, -1)];
        s2 = d == 0 ? pair : s2 + pair;
    }
    double inv_dx2 = 1.0 / (p->dx * p->dx);
    return (s2 - (double)(2 * p->dims) * f[s]) * inv_dx2;
}

/* a^beta dV/dphi = cV phi (phi^2/phi0^2 - 1) */
static double force(const orc_params* p, double cV, double phi)
{
    double inv_phi0sq = 1.0 / (p->phi0 * p->phi0);
    return (cV * phi) * ((phi * phi) * inv_phi0sq - 1.0);
}

/* d/dphi of force(): cV (3 phi^2/phi0^2 - 1) */
static double force_prime(const orc_params* p, double cV, double phi)
{
    double inv_phi0sq = 1.0 / (p->phi0 * p->phi0);
    return cV * (3.0 * (phi * phi) * inv_phi0sq - 1.0);
}

/* One leapfrog step n of Eqs. 3-5 (Jacobi: every site reads the old arrays). */
static void one_step(const orc_params* p, int64_t n, const double* phi, const double* v, double* phi_new,
                     double* v_new)
{
    double c[5];
    orc_coeffs(p, n, c);
    int64_t S = orc_sites(p);
    for (int64_t s = 0; s < S; ++s) {
        double lap = laplacian(p, phi, s);                           /* Eq. 3 */
        double vn = c[0] * v[s] + c[1] * (lap - force(p, c[2], phi[s])); /* Eq. 4 */
        v_new[s] = vn;
        phi_new[s] = phi[s] + p->deta * vn;                           /* Eq. 5 */
    }
}

/* Advance (phi, v) in place from step n0 through nsteps leapfrog steps.
 * Returns 0, or -1 when memory runs out. */
int orc_step(const orc_params* p, int64_t n0, int64_t nsteps, double* phi, double* v)
{
    int64_t S = orc_sites(p);
    double* phi_new = (double*)malloc((size_t)S * sizeof(double));
    double* v_new = (double*)malloc((size_t)S * sizeof(double));
    if (!phi_new || !v_new) {
        free(phi_new);
        free(v_new);
        return -1;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        one_step(p, n0 + k, phi, v, phi_new, v_new);
        memcpy(phi, phi_new, (size_t)S * sizeof(double));
        memcpy(v, v_new, (size_t)S * sizeof(double));
    }
    free(phi_new);
    free(v_new);
    return 0;
}

/* --------------------------------------------------------------- diagnostics */

static int negative(double f) { return f < 0.0; }

/* Eq. 7 weight of the link (s, t = s + e_d): |g| / sum_i |g_i| with g the
 * gradient at the link midpoint. */
static double link_weight(const orc_params* p, const double* phi, int64_t s, int64_t t, int d)
{
    double num = 0.0, den = 0.0;
    for (int e = 0; e < p->dims; ++e) {
        double g;
        if (e == d) {
            g = phi[t] - phi[s];
        } else {
            double gs = phi[neighbour(p, s, e, +1)] - phi[neighbour(p, s, e, -1)];
            double gt = phi[neighbour(p, t, e, +1)] - phi[neighbour(p, t, e, -1)];
            g = 0.25 * (gs + gt);
        }
        num += g * g;
        den += fabs(g);
    }
    return sqrt(num) / den;
}

static double potential(const orc_params* p, double phi)
{
    double u = phi * phi / (p->phi0 * p->phi0) - 1.0;
    return orc_V0(p) * u * u;
}

/* Eq. 7 and Eq. 8 on the field phi^n with the stored velocity dphi^{n-1/2}. */
void orc_measure(const orc_params* p, const double* phi, const double* v, orc_diag* out)
{
    int64_t S = orc_sites(p);
    double sum_w = 0.0, sum_ratio = 0.0;
    int64_t n_links = 0, n_wall = 0, n_vzero = 0, n_nonfinite = 0;
    for (int64_t s = 0; s < S; ++s) {
        if (!isfinite(phi[s]) || !isfinite(v[s])) ++n_nonfinite;
        /* links (s, s + e_d): each link of the periodic lattice exactly once */
        for (int d = 0; d < p->dims; ++d) {
            int64_t t = neighbour(p, s, d, +1);
            if (negative(phi[s]) != negative(phi[t])) {
                ++n_links;
                sum_w += link_weight(p, phi, s, t, d);
            }
        }
        /* wall sites: some nearest neighbour has the opposite sign */
        int wall = 0;
        for (int d = 0; d < p->dims; ++d)
            for (int step = -1; step <= 1; step += 2)
                if (negative(phi[neighbour(p, s, d, step)]) != negative(phi[s])) wall = 1;
        if (wall) {
            ++n_wall;
            double V = potential(p, phi[s]);
            if (V > 0.0)
                sum_ratio += v[s] * v[s] / V;
            else
                ++n_vzero;
        }
    }
    out->sum_w = sum_w;
    out->sum_ratio = sum_ratio;
    out->n_links = n_links;
    out->n_wall = n_wall;
    out->n_vzero = n_vzero;
    out->n_nonfinite = n_nonfinite;
    /* dA / V = dx^(D-1) / (S dx^D) = 1 / (S dx) */
    out->area_per_volume = sum_w / ((double)S * p->dx);
    int64_t nw = n_wall - n_vzero;
    out->gamma_v = nw > 0 ? sqrt(sum_ratio / (2.0 * (double)nw)) : 0.0;
}

/* ------------------------------------------------------- smooth observables */

/* obs 0: J = 1/2 sum_s sum_d ((phi_{s+e_d} - phi_s)/dx)^2    (gradient energy)
 * obs 1: J = dA/V sum_links (1 - sigma_s sigma_t)/2, sigma = tanh(phi/eps)
 *        (a smooth stand-in for the link count of Eq. 7). */
double orc_observable(const orc_params* p, int obs, double eps, const double* phi)
{
    int64_t S = orc_sites(p);
    double J = 0.0;
    for (int64_t s = 0; s < S; ++s)
        for (int d = 0; d < p->dims; ++d) {
            int64_t t = neighbour(p, s, d, +1);
            if (obs == 0) {
                double g = (phi[t] - phi[s]) / p->dx;
                J += 0.5 * g * g;
            } else {
                J += 0.5 * (1.0 - tanh(phi[s] / eps) * tanh(phi[t] / eps));
            }
        }
    if (obs == 1) J = J / ((double)S * p->dx);
    return J;
}

/* Gradient of orc_observable with respect to phi, written into g. */
void orc_observable_grad(const orc_params* p, int obs, double eps, const double* phi, double* g)
{
    int64_t S = orc_sites(p);
    for (int64_t s = 0; s < S; ++s) g[s] = 0.0;
    for (int64_t s = 0; s < S; ++s)
        for (int d = 0; d < p->dims; ++d) {
            int64_t t = neighbour(p, s, d, +1);
            if (obs == 0) {
                double dd = (phi[t] - phi[s]) / (p->dx * p->dx);
                g[t] += dd;
                g[s] -= dd;
            } else {
                double ss = tanh(phi[s] / eps), st = tanh(phi[t] / eps);
                double c = 1.0 / ((double)S * p->dx);
                g[s] += -0.5 * c * (1.0 - ss * ss) / eps * st;
                g[t] += -0.5 * c * (1.0 - st * st) / eps * ss;
            }
        }
}

/* ------------------------------------------------------------------ adjoint */

/* Gradient of J(phi^{n0+nsteps}) with respect to the initial state and alpha.
 * Every intermediate state is stored (plain, memory-hungry, for small boxes).
 * Outputs: *J, *dJ_dalpha, dJ_dphi[S], dJ_dv[S].  Returns 0, or -1 on no memory. */
int orc_adjoint(const orc_params* p, int64_t n0, int64_t nsteps, int obs, double eps, const double* phi_init,
                const double* v_init, double* J, double* dJ_dalpha, double* dJ_dphi, double* dJ_dv)
{
    int64_t S = orc_sites(p);
    size_t bytes = (size_t)S * sizeof(double);
    double* phis = (double*)malloc(bytes * (size_t)(nsteps + 1));
    double* vs = (double*)malloc(bytes * (size_t)(nsteps + 1));
    double* lt = (double*)malloc(bytes);
    double* lphi = (double*)malloc(bytes);
    double* lv = (double*)malloc(bytes);
    if (!phis || !vs || !lt || !lphi || !lv) {
        free(phis), free(vs), free(lt), free(lphi), free(lv);
        return -1;
    }
    memcpy(phis, phi_init, bytes);
    memcpy(vs, v_init, bytes);
    for (int64_t k = 0; k < nsteps; ++k)
        one_step(p, n0 + k, phis + k * S, vs + k * S, phis + (k + 1) * S, vs + (k + 1) * S);

    const double* phi_end = phis + nsteps * S;
    *J = orc_observable(p, obs, eps, phi_end);
    orc_observable_grad(p, obs, eps, phi_end, lphi);
    for (int64_t s = 0; s < S; ++s) lv[s] = 0.0;

    double dalpha = 0.0;
    for (int64_t k = nsteps - 1; k >= 0; --k) {
        const double* phi = phis + k * S;
        const double* v = vs + k * S;
        double c[5];
        orc_coeffs(p, n0 + k, c);
        double opd = 1.0 + c[3];
        double dc1 = -2.0 / (opd * opd) * c[4];     /* dc1/dalpha */
        double dc2 = -p->deta / (opd * opd) * c[4]; /* dc2/dalpha */
        for (int64_t s = 0; s < S; ++s) lt[s] = lv[s] + p->deta * lphi[s];
        for (int64_t s = 0; s < S; ++s) {
            double r = laplacian(p, phi, s) - force(p, c[2], phi[s]);
            dalpha += lt[s] * (dc1 * v[s] + dc2 * r);
        }
        for (int64_t s = 0; s < S; ++s) {
            lphi[s] = lphi[s] + c[1] * (laplacian(p, lt, s) - force_prime(p, c[2], phi[s]) * lt[s]);
            lv[s] = c[0] * lt[s];
        }
    }
    *dJ_dalpha = dalpha;
    memcpy(dJ_dphi, lphi, bytes);
    memcpy(dJ_dv, lv, bytes);
    free(phis), free(vs), free(lt), free(lphi), free(lv);
    return 0;
}
