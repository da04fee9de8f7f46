/*
 * FP64 CPU oracle of the Shan-Chen multiphase lattice Boltzmann time step
 * (arXiv 2506.17713, JAX-LaB, Section 2: Eqs. lbe, lbe_steps, collision_model,
 * macroeq, edm, mcmp_lbe, macroeq_mcp, eos_potential, software_ff_force_mcmp,
 * improved_virtual_density).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. The CUDA product path
 * never calls it and shares no code, header, table or constant with it.
 *
 * It is written to be read against the paper, not to be fast:
 *   - populations are array-of-structures, f[(k*N + n)*Q + i], n = x + nx*(y + ny*z);
 *   - the velocity set is enumerated from its definition (all e in {-1,0,1}^d
 *     with |e|^2 <= 2), weights follow from |e|^2;
 *   - the MRT matrix is built from the moment polynomials and inverted by
 *     Gauss-Jordan elimination; collision is a dense matrix-vector product;
 *   - streaming PUSHES post-collision populations into a second array;
 *   - every floating-point quantity is double; build with -ffp-contract=off;
 *   - reductions run sequentially in node order.
 * OpenMP only splits loops whose iterations write disjoint memory, so results
 * do not depend on the thread count.
 *
 * Readings of the paper taken where it is silent (same readings as the CUDA path):
 *   G_i = w_i / c_s^2 on all Q-1 links (so sum_i G_i e_i e_i = I);
 *   U^k = alpha p_EOS - c_s^2 rho for the EOS pseudopotential, U = g_kk psi^2/2 otherwise;
 *   psi = sqrt(max(0, 2 U / g_kk)) (argument clamped at zero, and U = 0 there);
 *   equilibrium velocity = bare sum_i f_i e_i / rho (per component, or the
 *   common Shan-Chen velocity when requested); EDM shift dU = F / rho;
 *   output velocity (sum_i f_i e_i + F/2) / rho;
 *   halfway bounce-back at solid nodes and WALL faces; solid nodes carry no
 *   populations; forces act on fluid nodes only;
 *   off-domain neighbours across a non-periodic face take the value at the
 *   coordinate-clamped in-domain node;
 *   rho_s = phi * rho_ave - drho, clamped to [rho_lo, rho_hi];
 *   constant-density x faces use the Zou-He / Hecht-Harting closure with zero
 *   tangential velocity, applied to the post-stream populations;
 *   body forces are accelerations: F_body^k = rho^k a^k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 19

enum { ORC_BGK = 0, ORC_MRT = 1 };
enum { ORC_PSI_EOS = 0, ORC_PSI_RHO = 1, ORC_PSI_EXP = 2 };
enum { ORC_CS = 0, ORC_PR = 1, ORC_VDW = 2, ORC_RK = 3, ORC_RKS = 4 };
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_PRESSURE = 2 };

typedef struct {
    int dim; /* 2 -> D2Q9, 3 -> D3Q19 */
    int nx, ny, nz;
    int ncomp;
    int collision;
    int common_velocity;
    double tau[2];
    double mrt_rates[2][19];
    int psi_kind[2];
    int eos[2];
    double eos_a[2], eos_b[2], eos_R[2], eos_omega[2], T_red[2];
    double alpha[2];
    double A[2];
    double g[2][2];
    double wet_phi[2], wet_drho[2], rho_lo[2], rho_hi[2];
    double accel[2][3];
    int face_bc[6]; /* -x, +x, -y, +y, -z, +z */
    double face_rho[6][2];
    double kappa[2];  /* surface-tension adjustment (Section 2.3, D2Q9 MRT only); 0 = off */
    int forcing;      /* ORC_FORCE_EDM (Eq. edm) | ORC_FORCE_MOMENT (F_m inside Eq. mrt_surface) */
} orc_params;

enum { ORC_FORCE_EDM = 0, ORC_FORCE_MOMENT = 1 };

typedef struct {
    orc_params p;
    int Q;
    int e[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    int opp[ORC_MAXQ];
    double M[ORC_MAXQ][ORC_MAXQ];
    double Minv[ORC_MAXQ][ORC_MAXQ];
    double rates[2][ORC_MAXQ];
    double T[2], alphaT[2]; /* absolute temperature and alpha(T) per component */
    long N;
    int dims[3];
    double *f, *fnew, *fpost;
    uint8_t *solid;   /* 1 = solid */
    uint8_t *bsolid;  /* 1 = solid with at least one fluid neighbour */
    double *rho, *j, *psi, *U, *F; /* rho/psi/U: [k][n]; j/F: [k][n][3] */
    long steps;
} orc_sim;

/* ------------------------------------------------------------------------ */
/* Equations of state (Section 2.2; the paper takes the forms and parameters  */
/* of Yuan & Schaefer 2006). T = T_red * Tc.                                 */
/* ------------------------------------------------------------------------ */

/* Pressure at absolute temperature T; the PR/RKS attraction factor alpha(T)
 * is passed in (it equals 1 at the critical temperature). */
static double eos_p_T(int eos, double a, double b, double R, double T, double alpha_T, double rho)
{
    switch (eos) {
    case ORC_CS: {
        double eta = b * rho / 4.0;
        double num = 1.0 + eta + eta * eta - eta * eta * eta;
        double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
        return rho * R * T * num / den - a * rho * rho;
    }
    case ORC_PR:
        return rho * R * T / (1.0 - b * rho)
               - a * alpha_T * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    case ORC_VDW:
        return rho * R * T / (1.0 - b * rho) - a * rho * rho;
    case ORC_RK:
        return rho * R * T / (1.0 - b * rho) - a * rho * rho / (sqrt(T) * (1.0 + b * rho));
    case ORC_RKS:
        return rho * R * T / (1.0 - b * rho) - a * alpha_T * rho * rho / (1.0 + b * rho);
    }
    return NAN;
}

static double eos_rho_pole(int eos, double b);

/* Critical temperature from its definition: the isotherm through the critical
 * point has a horizontal inflection, i.e. min_rho dp/drho = 0 there. Below Tc
 * the minimum slope is negative, above it positive; bisection on T, the inner
 * minimum by golden-section search on a central-difference slope. */
static double min_slope(int eos, double a, double b, double R, double T)
{
    double pole = eos_rho_pole(eos, b);
    double lo = 1e-6 * pole, hi = 0.999 * pole;
    /* coarse scan for the bracket of the minimum slope */
    const int ns = 2000;
    double best = INFINITY, rbest = lo;
    for (int m = 0; m <= ns; ++m) {
        double r = lo + (hi - lo) * m / ns, h = 1e-6 * r;
        double s = (eos_p_T(eos, a, b, R, T, 1.0, r + h) - eos_p_T(eos, a, b, R, T, 1.0, r - h)) / (2 * h);
        if (s < best) { best = s; rbest = r; }
    }
    double l = rbest - (hi - lo) / ns, u = rbest + (hi - lo) / ns;
    if (l < lo) l = lo;
    const double gr = 0.6180339887498949;
    for (int it = 0; it < 200 && u - l > 1e-14 * u; ++it) {
        double x1 = u - gr * (u - l), x2 = l + gr * (u - l);
        double h1 = 1e-5 * x1, h2 = 1e-5 * x2;
        double s1 = (eos_p_T(eos, a, b, R, T, 1.0, x1 + h1) - eos_p_T(eos, a, b, R, T, 1.0, x1 - h1)) / (2 * h1);
        double s2 = (eos_p_T(eos, a, b, R, T, 1.0, x2 + h2) - eos_p_T(eos, a, b, R, T, 1.0, x2 - h2)) / (2 * h2);
        if (s1 < s2) u = x2; else l = x1;
    }
    double r = 0.5 * (l + u), h = 1e-5 * r;
    return (eos_p_T(eos, a, b, R, T, 1.0, r + h) - eos_p_T(eos, a, b, R, T, 1.0, r - h)) / (2 * h);
}

double orc_eos_Tc(int eos, double a, double b, double R)
{
    /* bracket: the critical temperature is of order a/(bR) for every EOS here
     * (RK: (a/(bR))^(2/3)) */
    double scale = eos == ORC_RK ? pow(a / (b * R), 2.0 / 3.0) : a / (b * R);
    double lo = 0.01 * scale, hi = 10.0 * scale;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double T = 0.5 * (lo + hi);
        if (min_slope(eos, a, b, R, T) < 0.0) lo = T; else hi = T;
    }
    return 0.5 * (lo + hi);
}

/* alpha(T) of PR / RKS at reduced temperature T_red (1 for the other EOS) */
static double eos_alpha(int eos, double omega, double T_red)
{
    if (eos != ORC_PR && eos != ORC_RKS) return 1.0;
    double m = eos == ORC_PR ? 0.37464 + 1.54226 * omega - 0.26992 * omega * omega
                             : 0.480 + 1.574 * omega - 0.176 * omega * omega;
    double s = 1.0 + m * (1.0 - sqrt(T_red));
    return s * s;
}

double orc_eos_pressure(int eos, double a, double b, double R, double omega,
                        double T_red, double rho)
{
    double T = T_red * orc_eos_Tc(eos, a, b, R);
    return eos_p_T(eos, a, b, R, T, eos_alpha(eos, omega, T_red), rho);
}

/* Upper end of the physical density range of an EOS (repulsive pole). */
static double eos_rho_pole(int eos, double b)
{
    return eos == ORC_CS ? 4.0 / b : 1.0 / b;
}

/* ------------------------------------------------------------------------ */
/* Pseudopotential (Eq. eos_potential and the psi = rho, psi = exp(-1/rho)   */
/* forms of Sections 3.3.2 and 5).                                           */
/* ------------------------------------------------------------------------ */

static const double CS2 = 1.0 / 3.0;

/* T[k], alphaT[k]: absolute temperature T_red * Tc and alpha(T) of component k */
static void psi_of_rho(const orc_params* p, const double* T, const double* alphaT, int k,
                       double rho, double* psi, double* U)
{
    double gkk = p->g[k][k];
    if (p->psi_kind[k] == ORC_PSI_EOS) {
        double pe = eos_p_T(p->eos[k], p->eos_a[k], p->eos_b[k], p->eos_R[k], T[k], alphaT[k], rho);
        double u = p->alpha[k] * pe - CS2 * rho;
        double arg = 2.0 * u / gkk;
        /* psi is real only where 2U/g >= 0; elsewhere psi = 0 and, keeping
         * U = g psi^2 / 2 as everywhere else, U = 0 */
        *U = arg > 0.0 ? u : 0.0;
        *psi = sqrt(arg > 0.0 ? arg : 0.0);
    } else {
        double s = p->psi_kind[k] == ORC_PSI_RHO ? rho : exp(-1.0 / rho);
        *psi = s;
        *U = 0.5 * gkk * s * s;
    }
}

/* Bulk pressure of a single component at uniform density: c_s^2 rho + U. */
static void temperatures(const orc_params* p, double* T, double* alphaT)
{
    for (int k = 0; k < 2; ++k) {
        T[k] = 0.0; alphaT[k] = 1.0;
        if (p->psi_kind[k] != ORC_PSI_EOS || k >= p->ncomp) continue;
        T[k] = p->T_red[k] * orc_eos_Tc(p->eos[k], p->eos_a[k], p->eos_b[k], p->eos_R[k]);
        alphaT[k] = eos_alpha(p->eos[k], p->eos_omega[k], p->T_red[k]);
    }
}

double orc_bulk_pressure(const orc_params* p, int k, double rho)
{
    double psi, U, T[2], aT[2];
    temperatures(p, T, aT);
    psi_of_rho(p, T, aT, k, rho, &psi, &U);
    return CS2 * rho + U;
}

/* ------------------------------------------------------------------------ */
/* Maxwell equal-area construction (coexistence densities, Section 3.1).      */
/* Finds rho_g < rho_l with p(rho_g) = p(rho_l) = p_s and                     */
/* int_{rho_g}^{rho_l} (p(rho) - p_s) / rho^2 drho = 0.                       */
/* ------------------------------------------------------------------------ */

typedef double (*pfun)(const void* ctx, double rho);

typedef struct { int eos; double a, b, R, T, alphaT; } eos_ctx;
static double p_eos(const void* c, double rho)
{
    const eos_ctx* e = (const eos_ctx*)c;
    return eos_p_T(e->eos, e->a, e->b, e->R, e->T, e->alphaT, rho);
}
typedef struct { const orc_params* p; int k; double T[2], aT[2]; } bulk_ctx;
static double p_bulk(const void* c, double rho)
{
    const bulk_ctx* b = (const bulk_ctx*)c;
    double psi, U;
    psi_of_rho(b->p, b->T, b->aT, b->k, rho, &psi, &U);
    return CS2 * rho + U;
}

/* root of p(rho) = ps on [lo, hi] where p - ps changes sign (bisection) */
static double bisect_root(pfun p, const void* c, double ps, double lo, double hi)
{
    double flo = p(c, lo) - ps;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = p(c, mid) - ps;
        if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi);
}

/* 10-point Gauss-Legendre nodes/weights on [-1, 1] (Abramowitz & Stegun 25.4.30) */
static const double GL_X[5] = {0.1488743389816312, 0.4333953941292472, 0.6794095682990244,
                               0.8650633666889845, 0.9739065285171717};
static const double GL_W[5] = {0.2955242247147529, 0.2692667193099963, 0.2190863625159820,
                               0.1494513491505806, 0.0666713443086881};

static double area(pfun p, const void* c, double ps, double rg, double rl)
{
    const int panels = 400;
    double h = (rl - rg) / panels, sum = 0.0;
    for (int m = 0; m < panels; ++m) {
        double mid = rg + (m + 0.5) * h, half = 0.5 * h;
        for (int q = 0; q < 5; ++q) {
            double r1 = mid - half * GL_X[q], r2 = mid + half * GL_X[q];
            sum += GL_W[q] * half * ((p(c, r1) - ps) / (r1 * r1) + (p(c, r2) - ps) / (r2 * r2));
        }
    }
    return sum;
}

/* golden-section search for an extremum of p on [lo, hi] (sign=+1 max, -1 min) */
static double golden(pfun p, const void* c, double lo, double hi, double sign)
{
    const double gr = 0.6180339887498949;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double f1 = sign * p(c, x1), f2 = sign * p(c, x2);
    for (int it = 0; it < 300 && hi - lo > 1e-15 * hi; ++it) {
        if (f1 > f2) { hi = x2; x2 = x1; f2 = f1; x1 = hi - gr * (hi - lo); f1 = sign * p(c, x1); }
        else { lo = x1; x1 = x2; f1 = f2; x2 = lo + gr * (hi - lo); f2 = sign * p(c, x2); }
    }
    return 0.5 * (lo + hi);
}

static int maxwell_generic(pfun p, const void* c, double rmin, double rmax,
                           double* rho_g, double* rho_l, double* p_sat)
{
    /* locate the van der Waals loop: first local max then local min of p */
    const int ns = 20000;
    double lr0 = log(rmin), lr1 = log(rmax);
    double prev = p(c, rmin), rprev = rmin;
    double ra = -1.0, rb = -1.0;
    int rising = 1;
    for (int m = 1; m <= ns; ++m) {
        double r = exp(lr0 + (lr1 - lr0) * m / ns);
        double v = p(c, r);
        if (rising && v < prev && ra < 0) {
            double lo = exp(lr0 + (lr1 - lr0) * (m - 2 > 0 ? m - 2 : 0) / ns);
            ra = golden(p, c, lo, r, +1.0);
            rising = 0;
        } else if (!rising && v > prev && rb < 0) {
            double lo = exp(lr0 + (lr1 - lr0) * (m - 2 > 0 ? m - 2 : 0) / ns);
            rb = golden(p, c, lo, r, -1.0);
            break;
        }
        prev = v; rprev = r;
    }
    (void)rprev;
    if (ra < 0 || rb < 0) return -1; /* supercritical: no loop */
    double pmax = p(c, ra), pmin = p(c, rb);
    double lo = pmin > 0.0 ? pmin : 0.0, hi = pmax;
    double rg = 0, rl = 0, ps = 0;
    for (int it = 0; it < 200; ++it) {
        ps = 0.5 * (lo + hi);
        rg = bisect_root(p, c, ps, rmin, ra);
        rl = bisect_root(p, c, ps, rb, rmax);
        double A = area(p, c, ps, rg, rl);
        if (A > 0.0) lo = ps; else hi = ps; /* area decreases with p_s */
        if (hi - lo <= 1e-16 * hi) break;
    }
    *rho_g = rg; *rho_l = rl; if (p_sat) *p_sat = ps;
    return 0;
}

/* Coexistence densities of an EOS at T = T_red * Tc (Maxwell construction). */
int orc_maxwell_eos(int eos, double a, double b, double R, double omega, double T_red,
                    double* rho_g, double* rho_l, double* p_sat)
{
    eos_ctx c = {eos, a, b, R, T_red * orc_eos_Tc(eos, a, b, R), eos_alpha(eos, omega, T_red)};
    double pole = eos_rho_pole(eos, b);
    return maxwell_generic(p_eos, &c, 1e-8 * pole, (1.0 - 1e-9) * pole, rho_g, rho_l, p_sat);
}

/* Coexistence of the model's own bulk pressure c_s^2 rho + U(rho) of component k
 * (for psi = exp(-1/rho) this is the thermodynamically consistent pair). */
int orc_maxwell_bulk(const orc_params* p, int k, double rmin, double rmax,
                     double* rho_g, double* rho_l, double* p_sat)
{
    bulk_ctx c;
    c.p = p; c.k = k;
    temperatures(p, c.T, c.aT);
    return maxwell_generic(p_bulk, &c, rmin, rmax, rho_g, rho_l, p_sat);
}

/* ------------------------------------------------------------------------ */
/* Lattice: velocity set, weights, MRT moment basis                           */
/* ------------------------------------------------------------------------ */

static void build_lattice(orc_sim* s)
{
    int d = s->p.dim, q = 0;
    for (int c = -1; c <= 1; ++c) /* z (only 0 in 2D) */
        for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a) {
                if (d == 2 && c != 0) continue;
                int e2 = a * a + b * b + c * c;
                if (e2 > 2) continue;
                s->e[q][0] = a; s->e[q][1] = b; s->e[q][2] = c;
                if (d == 2) s->w[q] = e2 == 0 ? 4.0 / 9.0 : (e2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
                else s->w[q] = e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++q;
            }
    s->Q = q;
    for (int i = 0; i < q; ++i)
        for (int m = 0; m < q; ++m)
            if (s->e[m][0] == -s->e[i][0] && s->e[m][1] == -s->e[i][1] && s->e[m][2] == -s->e[i][2])
                s->opp[i] = m;
}

/* Moment a of velocity e: the Gram-Schmidt polynomials of Lallemand & Luo (D2Q9)
 * and d'Humieres et al. 2002 (D3Q19), in their standard order. */
static double moment_poly(int dim, int a, const int* e)
{
    double x = e[0], y = e[1], z = e[2];
    double e2 = x * x + y * y + z * z;
    if (dim == 2) {
        switch (a) {
        case 0: return 1.0;
        case 1: return -4.0 + 3.0 * e2;
        case 2: return 4.0 - 10.5 * e2 + 4.5 * e2 * e2;
        case 3: return x;
        case 4: return (-5.0 + 3.0 * e2) * x;
        case 5: return y;
        case 6: return (-5.0 + 3.0 * e2) * y;
        case 7: return x * x - y * y;
        case 8: return x * y;
        }
    } else {
        switch (a) {
        case 0: return 1.0;
        case 1: return 19.0 * e2 - 30.0;
        case 2: return (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * e2 - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * e2 - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * e2 - 9.0) * z;
        case 9: return 3.0 * x * x - e2;
        case 10: return (3.0 * e2 - 5.0) * (3.0 * x * x - e2);
        case 11: return y * y - z * z;
        case 12: return (3.0 * e2 - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        case 18: return (x * x - y * y) * z;
        }
    }
    return 0.0;
}

/* Gauss-Jordan inversion with partial pivoting; returns 0 on success. */
static int invert(int n, double A[ORC_MAXQ][ORC_MAXQ], double Ainv[ORC_MAXQ][ORC_MAXQ])
{
    double a[ORC_MAXQ][2 * ORC_MAXQ];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) a[r][c] = c < n ? A[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (fabs(a[piv][c]) < 1e-300) return -1;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) { double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
        double d = a[c][c];
        for (int k = 0; k < 2 * n; ++k) a[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = a[r][c];
            if (m != 0.0) for (int k = 0; k < 2 * n; ++k) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < n; ++r) for (int c = 0; c < n; ++c) Ainv[r][c] = a[r][c + n];
    return 0;
}

/* stress moments take 1/tau, conserved moments take 0, the rest the given rates */
static int is_stress(int dim, int a)
{
    if (dim == 2) return a == 7 || a == 8;
    return a == 9 || a == 11 || a == 13 || a == 14 || a == 15;
}
static int is_conserved(int dim, int a)
{
    if (dim == 2) return a == 0 || a == 3 || a == 5;
    return a == 0 || a == 3 || a == 5 || a == 7;
}

static int build_mrt(orc_sim* s)
{
    int Q = s->Q, d = s->p.dim;
    for (int a = 0; a < Q; ++a)
        for (int i = 0; i < Q; ++i) s->M[a][i] = moment_poly(d, a, s->e[i]);
    if (invert(Q, s->M, s->Minv)) return -1;
    for (int k = 0; k < 2; ++k)
        for (int a = 0; a < Q; ++a) {
            if (is_conserved(d, a)) s->rates[k][a] = 0.0;
            else if (is_stress(d, a)) s->rates[k][a] = 1.0 / s->p.tau[k];
            else s->rates[k][a] = s->p.mrt_rates[k][a];
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */

static inline long node_of(const orc_sim* s, int x, int y, int z)
{
    return (long)x + (long)s->dims[0] * ((long)y + (long)s->dims[1] * (long)z);
}
static inline void coords_of(const orc_sim* s, long n, int* c)
{
    c[0] = (int)(n % s->dims[0]);
    c[1] = (int)((n / s->dims[0]) % s->dims[1]);
    c[2] = (int)(n / ((long)s->dims[0] * s->dims[1]));
}

/* Neighbour for the force and virtual-density stencils: periodic faces wrap,
 * non-periodic faces clamp the coordinate into the domain. */
static long stencil_neighbour(const orc_sim* s, const int* c, const int* e)
{
    int t[3];
    for (int a = 0; a < 3; ++a) {
        int v = c[a] + e[a], n = s->dims[a];
        if (v < 0) v = s->p.face_bc[2 * a] == ORC_PERIODIC ? v + n : 0;
        else if (v >= n) v = s->p.face_bc[2 * a + 1] == ORC_PERIODIC ? v - n : n - 1;
        t[a] = v;
    }
    return node_of(s, t[0], t[1], t[2]);
}

/* Streaming target of (node c, direction e).
 * returns 0: regular target in *out; 1: bounce back; 2: leaves through a pressure face */
static int stream_target(const orc_sim* s, const int* c, const int* e, long* out)
{
    int t[3], wall = 0;
    /* the x faces are checked first so that a pressure face wins over a wall */
    for (int a = 0; a < 3; ++a) {
        int v = c[a] + e[a], n = s->dims[a];
        int face = v < 0 ? 2 * a : (v >= n ? 2 * a + 1 : -1);
        if (face >= 0) {
            int bc = s->p.face_bc[face];
            if (bc == ORC_PRESSURE) return 2;
            if (bc == ORC_WALL) wall = 1;
            v = v < 0 ? v + n : v - n;
        }
        t[a] = v;
    }
    if (wall) return 1;
    long m = node_of(s, t[0], t[1], t[2]);
    if (s->solid[m]) return 1;
    *out = m;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Creation                                                                  */
/* ------------------------------------------------------------------------ */

orc_sim* orc_create(const orc_params* p)
{
    if (!p || (p->dim != 2 && p->dim != 3) || p->ncomp < 1 || p->ncomp > 2) return NULL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->dim == 2 && p->nz != 1)) return NULL;
    if (p->forcing != ORC_FORCE_EDM && p->forcing != ORC_FORCE_MOMENT) return NULL;
    /* a 2-D lattice has no z velocity: a z acceleration is refused, not carried in u.u */
    if (p->dim == 2 && (p->accel[0][2] != 0.0 || p->accel[1][2] != 0.0)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->dims[0] = p->nx; s->dims[1] = p->ny; s->dims[2] = p->nz;
    s->N = (long)p->nx * p->ny * p->nz;
    build_lattice(s);
    if (build_mrt(s)) { free(s); return NULL; }
    temperatures(p, s->T, s->alphaT);
    long K = p->ncomp, N = s->N, Q = s->Q;
    s->f = (double*)calloc((size_t)(K * N * Q), sizeof(double));
    s->fnew = (double*)calloc((size_t)(K * N * Q), sizeof(double));
    s->fpost = (double*)calloc((size_t)(K * N * Q), sizeof(double));
    s->solid = (uint8_t*)calloc((size_t)N, 1);
    s->bsolid = (uint8_t*)calloc((size_t)N, 1);
    s->rho = (double*)calloc((size_t)(K * N), sizeof(double));
    s->psi = (double*)calloc((size_t)(K * N), sizeof(double));
    s->U = (double*)calloc((size_t)(K * N), sizeof(double));
    s->j = (double*)calloc((size_t)(K * N * 3), sizeof(double));
    s->F = (double*)calloc((size_t)(K * N * 3), sizeof(double));
    if (!s->f || !s->fnew || !s->fpost || !s->solid || !s->bsolid || !s->rho || !s->psi ||
        !s->U || !s->j || !s->F) {
        free(s->f); free(s->fnew); free(s->fpost); free(s->solid); free(s->bsolid);
        free(s->rho); free(s->psi); free(s->U); free(s->j); free(s->F); free(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->f); free(s->fnew); free(s->fpost); free(s->solid); free(s->bsolid);
    free(s->rho); free(s->psi); free(s->U); free(s->j); free(s->F);
    free(s);
}

int orc_Q(const orc_sim* s) { return s->Q; }
long orc_steps(const orc_sim* s) { return s->steps; }
void orc_velocity_set(const orc_sim* s, int* e, double* w)
{
    for (int i = 0; i < s->Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = s->e[i][a];
        w[i] = s->w[i];
    }
}
void orc_mrt_matrices(const orc_sim* s, double* M, double* Minv)
{
    for (int a = 0; a < s->Q; ++a)
        for (int i = 0; i < s->Q; ++i) { M[a * s->Q + i] = s->M[a][i]; Minv[a * s->Q + i] = s->Minv[a][i]; }
}
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_geometry(orc_sim* s, const uint8_t* solid)
{
    long N = s->N;
    for (long n = 0; n < N; ++n) s->solid[n] = solid ? (solid[n] != 0) : 0;
    /* boundary solids: solids with a fluid node among their Q-1 stencil neighbours */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int c[3];
        s->bsolid[n] = 0;
        if (!s->solid[n]) continue;
        coords_of(s, n, c);
        for (int i = 0; i < s->Q; ++i) {
            if (s->e[i][0] == 0 && s->e[i][1] == 0 && s->e[i][2] == 0) continue;
            if (!s->solid[stencil_neighbour(s, c, s->e[i])]) { s->bsolid[n] = 1; break; }
        }
    }
}

static void pressure_faces_on(orc_sim* s, double* farr, int k0, int k1);

/* f^eq_i(rho, u) = w_i rho (1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2)) */
static double feq(const orc_sim* s, int i, double rho, const double* u)
{
    double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return s->w[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Post-stream populations := f^eq(rho, u) at fluid nodes (u may be NULL = rest),
 * then the constant-density face closure, like every post-stream state.
 * u is laid out [dim][N]. */
void orc_init_fields(orc_sim* s, int k, const double* rho, const double* u)
{
    long N = s->N;
    int Q = s->Q, d = s->p.dim;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double* fn = s->f + ((long)k * N + n) * Q;
        if (s->solid[n]) { for (int i = 0; i < Q; ++i) fn[i] = 0.0; continue; }
        double v[3] = {0, 0, 0};
        if (u) for (int a = 0; a < d; ++a) v[a] = u[(long)a * N + n];
        for (int i = 0; i < Q; ++i) fn[i] = feq(s, i, rho[n], v);
    }
    pressure_faces_on(s, s->f, k, k + 1);
    s->steps = 0;
}

/* Post-stream populations given directly, [Q][N] in the oracle's velocity order
 * (the constant-density face closure is applied to them). */
void orc_set_populations(orc_sim* s, int k, const double* fin)
{
    long N = s->N;
    int Q = s->Q;
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < Q; ++i)
            s->f[((long)k * N + n) * Q + i] = s->solid[n] ? 0.0 : fin[(long)i * N + n];
    pressure_faces_on(s, s->f, k, k + 1);
}
void orc_get_populations(const orc_sim* s, int k, double* fout)
{
    long N = s->N;
    int Q = s->Q;
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < Q; ++i) fout[(long)i * N + n] = s->f[((long)k * N + n) * Q + i];
}

/* ------------------------------------------------------------------------ */
/* Step pieces                                                               */
/* ------------------------------------------------------------------------ */

/* (1) rho^k = sum_i f_i^k, j^k = sum_i f_i^k e_i at fluid nodes (Eq. macroeq_mcp) */
static void moments(orc_sim* s)
{
    long N = s->N;
    int Q = s->Q, K = s->p.ncomp;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        for (int k = 0; k < K; ++k) {
            double r = 0, jx = 0, jy = 0, jz = 0;
            if (!s->solid[n]) {
                const double* fn = s->f + ((long)k * N + n) * Q;
                for (int i = 0; i < Q; ++i) {
                    r += fn[i];
                    jx += fn[i] * s->e[i][0]; jy += fn[i] * s->e[i][1]; jz += fn[i] * s->e[i][2];
                }
            }
            s->rho[(long)k * N + n] = r;
            double* jn = s->j + ((long)k * N + n) * 3;
            jn[0] = jx; jn[1] = jy; jn[2] = jz;
        }
    }
}

/* (2) improved virtual density at boundary solids (Eq. improved_virtual_density):
 * rho_ave = sum_j w_j rho(x_s + e_j) over fluid neighbours / sum_j w_j over the same;
 * rho_s = phi rho_ave - drho, limited to [rho_lo, rho_hi]. */
static void virtual_density(orc_sim* s)
{
    long N = s->N;
    int Q = s->Q, K = s->p.ncomp;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (!s->bsolid[n]) continue;
        int c[3];
        coords_of(s, n, c);
        for (int k = 0; k < K; ++k) {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < Q; ++i) {
                if (s->e[i][0] == 0 && s->e[i][1] == 0 && s->e[i][2] == 0) continue;
                long m = stencil_neighbour(s, c, s->e[i]);
                if (s->solid[m]) continue;
                num += s->w[i] * s->rho[(long)k * N + m];
                den += s->w[i];
            }
            double r = s->p.wet_phi[k] * (num / den) - s->p.wet_drho[k];
            if (r < s->p.rho_lo[k]) r = s->p.rho_lo[k];
            if (r > s->p.rho_hi[k]) r = s->p.rho_hi[k];
            s->rho[(long)k * N + n] = r;
        }
    }
}

/* (3) psi^k and U^k at fluid and boundary-solid nodes (Eq. eos_potential) */
static void pseudopotential(orc_sim* s)
{
    long N = s->N;
    int K = s->p.ncomp;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        for (int k = 0; k < K; ++k) {
            double ps = 0.0, U = 0.0;
            if (!s->solid[n] || s->bsolid[n]) psi_of_rho(&s->p, s->T, s->alphaT, k, s->rho[(long)k * N + n], &ps, &U);
            s->psi[(long)k * N + n] = ps;
            s->U[(long)k * N + n] = U;
        }
    }
}

/* (4) interaction force from given psi/U fields (Eq. software_ff_force_mcmp)
 *   F_SC^k = -psi^k(x) sum_k' g_kk' sum_i G_i psi^k'(x + e_i) e_i
 *   F_ZC^k = -sum_i G_i U^k(x + e_i) e_i,   G_i = w_i / c_s^2
 *   F^k = A_kk F_ZC^k + (1 - A_kk) F_SC^k   (+ rho^k a^k when with_body)
 * psi, U: [K][N]; F out: [K][N][3]; evaluated at fluid nodes, zero at solids. */
void orc_interaction_force(const orc_sim* s, const double* psi, const double* U,
                           const double* rho, int with_body, double* F)
{
    long N = s->N;
    int Q = s->Q, K = s->p.ncomp;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int c[3];
        coords_of(s, n, c);
        for (int k = 0; k < K; ++k) {
            double* Fn = F + ((long)k * N + n) * 3;
            Fn[0] = Fn[1] = Fn[2] = 0.0;
            if (s->solid[n]) continue;
            double sc[3] = {0, 0, 0}, zc[3] = {0, 0, 0};
            for (int i = 0; i < Q; ++i) {
                if (s->e[i][0] == 0 && s->e[i][1] == 0 && s->e[i][2] == 0) continue;
                long m = stencil_neighbour(s, c, s->e[i]);
                double G = s->w[i] / CS2;
                double acc = 0.0;
                for (int kp = 0; kp < K; ++kp) acc += s->p.g[k][kp] * psi[(long)kp * N + m];
                for (int a = 0; a < 3; ++a) {
                    sc[a] += G * acc * s->e[i][a];
                    zc[a] += G * U[(long)k * N + m] * s->e[i][a];
                }
            }
            double A = s->p.A[k], pk = psi[(long)k * N + n];
            for (int a = 0; a < 3; ++a) {
                Fn[a] = A * (-zc[a]) + (1.0 - A) * (-pk * sc[a]);
                if (with_body) Fn[a] += rho[(long)k * N + n] * s->p.accel[k][a];
            }
        }
    }
}

/* the full pipeline up to the force at the current time level */
static void fields_and_force(orc_sim* s)
{
    moments(s);
    virtual_density(s);
    pseudopotential(s);
    orc_interaction_force(s, s->psi, s->U, s->rho, 1, s->F);
}

/* Source term C of the surface-tension adjustment (Section 2.3, Eq. mrt_surface and
 * Eq. li_surface_adjust), D2Q9 moment order (rho, e, eps, jx, qx, jy, qy, pxx, pxy):
 *   C = [0, 1.5 s_e (Qxx + Qyy), -1.5 s_eps (Qxx + Qyy), 0, 0, 0, 0, -s_nu (Qxx - Qyy), -s_nu Qxy]
 * with the pressure-tensor term
 *   Q = kappa (g_kk / 2) [ (1 - A) psi(x) sum_i G_i (psi(x + e_i) - psi(x)) e_i e_i
 *                          + (A / 2) sum_i G_i (psi(x + e_i)^2 - psi(x)^2) e_i e_i ],
 * G_i = w_i / c_s^2 the force weights. The factor g_kk / 2 is that of Li et al. (2013),
 * whose scheme the paper implements. Together with the moment-space forcing of the same
 * equation (ORC_FORCE_MOMENT) the surface tension scales with 1 - kappa as the paper states
 * (pinned by the Laplace tests); with EDM forcing the F F / rho stress of that scheme does
 * not scale with kappa. Zero unless D2Q9, MRT, kappa != 0. */
/* Q = (Qxx, Qyy, Qxy) at node n from the psi field psi [K][N] (Q as defined above) */
void orc_surface_Q(const orc_sim* s, const double* psi, long n, int k, double* Qout)
{
    int c[3];
    coords_of(s, n, c);
    const double px = psi[(long)k * s->N + n], A = s->p.A[k];
    double q[2][2] = {{0, 0}, {0, 0}};
    for (int i = 0; i < s->Q; ++i) {
        if (s->e[i][0] == 0 && s->e[i][1] == 0 && s->e[i][2] == 0) continue;
        const long m = stencil_neighbour(s, c, s->e[i]);
        const double pn = psi[(long)k * s->N + m];
        const double G = s->w[i] / CS2;
        const double t = (1.0 - A) * px * (pn - px) + 0.5 * A * (pn * pn - px * px);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) q[a][b] += G * t * s->e[i][a] * s->e[i][b];
    }
    const double f = s->p.kappa[k] * 0.5 * s->p.g[k][k];
    Qout[0] = f * q[0][0];
    Qout[1] = f * q[1][1];
    Qout[2] = f * q[0][1];
}

static void surface_source(const orc_sim* s, long n, int k, double* C)
{
    for (int a = 0; a < s->Q; ++a) C[a] = 0.0;
    if (s->p.dim != 2 || s->p.collision != ORC_MRT || s->p.kappa[k] == 0.0) return;
    double Q[3];
    orc_surface_Q(s, s->psi, n, k, Q);
    const double Qxx = Q[0], Qyy = Q[1], Qxy = Q[2];
    const double se = s->rates[k][1], seps = s->rates[k][2], snu = s->rates[k][7];
    C[1] = 1.5 * se * (Qxx + Qyy);
    C[2] = -1.5 * seps * (Qxx + Qyy);
    C[7] = -snu * (Qxx - Qyy);
    C[8] = -snu * Qxy;
}

/* Moment-space forcing, the F_m that Eq. mrt_surface places inside M^-1[...] with the
 * relaxation (Section 2.3; the scheme of Li et al. 2013 that the paper implements for
 * the surface-tension adjustment). It is the forcing of Guo et al. (2002) written in
 * moment space:
 *   v = u_eq + F / (2 rho)                         (equilibrium at the physical velocity)
 *   S_i = w_i [ (e_i - v) / c_s^2 + (e_i . v) e_i / c_s^4 ] . F
 *   m* = m - S (m - m^eq(rho, v)) + (I - S/2) M S_i + C,     f* = M^-1 m*
 * BGK is the case S = I / tau:  f* = f - (f - f^eq(rho, v)) / tau + (1 - 1/(2 tau)) S_i. */
static void collide_node_moment_forcing(const orc_sim* s, const double* fin, double rho, const double* ueq,
                                        const double* dU, int k, const double* Cm, double* fout)
{
    int Q = s->Q;
    double v[3], F[3];
    for (int a = 0; a < 3; ++a) { v[a] = ueq[a] + 0.5 * dU[a]; F[a] = rho * dU[a]; }
    double neq[ORC_MAXQ], Si[ORC_MAXQ];
    for (int i = 0; i < Q; ++i) {
        neq[i] = fin[i] - feq(s, i, rho, v);
        double ev = s->e[i][0] * v[0] + s->e[i][1] * v[1] + s->e[i][2] * v[2];
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) acc += ((s->e[i][a] - v[a]) / CS2 + ev * s->e[i][a] / (CS2 * CS2)) * F[a];
        Si[i] = s->w[i] * acc;
    }
    if (s->p.collision == ORC_BGK) {
        double tau = s->p.tau[k];
        for (int i = 0; i < Q; ++i) fout[i] = fin[i] - neq[i] / tau + (1.0 - 0.5 / tau) * Si[i];
        return;
    }
    double m[ORC_MAXQ];
    for (int a = 0; a < Q; ++a) {
        double mn = 0.0, ms = 0.0;
        for (int i = 0; i < Q; ++i) { mn += s->M[a][i] * neq[i]; ms += s->M[a][i] * Si[i]; }
        double sa = s->rates[k][a];
        /* m* - m = -s_a m_neq + (1 - s_a / 2) (M S)_a + C_a */
        m[a] = -sa * mn + (1.0 - 0.5 * sa) * ms + (Cm ? Cm[a] : 0.0);
    }
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int a = 0; a < Q; ++a) acc += s->Minv[i][a] * m[a];
        fout[i] = fin[i] + acc;
    }
}

/* (5)+(6) collision of one node, one component.
 * fin: Q post-stream populations; u_eq: equilibrium velocity; dU = F/rho;
 * Cm: moment-space source (MRT, may be NULL). */
static void collide_node(const orc_sim* s, const double* fin, double rho, const double* ueq,
                         const double* dU, int k, const double* Cm, double* fout)
{
    if (s->p.forcing == ORC_FORCE_MOMENT) {
        collide_node_moment_forcing(s, fin, rho, ueq, dU, k, Cm, fout);
        return;
    }
    int Q = s->Q;
    double fe[ORC_MAXQ], neq[ORC_MAXQ];
    for (int i = 0; i < Q; ++i) { fe[i] = feq(s, i, rho, ueq); neq[i] = fin[i] - fe[i]; }
    if (s->p.collision == ORC_BGK) {
        double om = 1.0 / s->p.tau[k];
        for (int i = 0; i < Q; ++i) fout[i] = fin[i] - om * neq[i];
    } else {
        double m[ORC_MAXQ];
        for (int a = 0; a < Q; ++a) {
            double acc = 0.0;
            for (int i = 0; i < Q; ++i) acc += s->M[a][i] * neq[i];
            m[a] = s->rates[k][a] * acc - (Cm ? Cm[a] : 0.0);   /* f* = f - M^-1 (S m_neq - C) */
        }
        for (int i = 0; i < Q; ++i) {
            double acc = 0.0;
            for (int a = 0; a < Q; ++a) acc += s->Minv[i][a] * m[a];
            fout[i] = fin[i] - acc;
        }
    }
    /* Exact Difference Method (Eq. edm) */
    double u2[3] = {ueq[0] + dU[0], ueq[1] + dU[1], ueq[2] + dU[2]};
    for (int i = 0; i < Q; ++i) fout[i] += feq(s, i, rho, u2) - feq(s, i, rho, ueq);
}

/* single-node collision for tests: f in, F in, f* out, using the node's own bare velocity */
void orc_collide_single(const orc_sim* s, int k, const double* fin, const double* F, double* fout)
{
    int Q = s->Q;
    double rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        rho += fin[i];
        for (int a = 0; a < 3; ++a) j[a] += fin[i] * s->e[i][a];
    }
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double dU[3] = {F[0] / rho, F[1] / rho, F[2] / rho};
    collide_node(s, fin, rho, u, dU, k, NULL, fout);
}

static void collide(orc_sim* s)
{
    long N = s->N;
    int Q = s->Q, K = s->p.ncomp;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->solid[n]) continue;
        double ucommon[3] = {0, 0, 0};
        if (s->p.common_velocity && K > 1) {
            double num[3] = {0, 0, 0}, den = 0.0;
            for (int k = 0; k < K; ++k) {
                const double* jn = s->j + ((long)k * N + n) * 3;
                for (int a = 0; a < 3; ++a) num[a] += jn[a] / s->p.tau[k];
                den += s->rho[(long)k * N + n] / s->p.tau[k];
            }
            for (int a = 0; a < 3; ++a) ucommon[a] = num[a] / den;
        }
        for (int k = 0; k < K; ++k) {
            double r = s->rho[(long)k * N + n];
            const double* jn = s->j + ((long)k * N + n) * 3;
            const double* Fn = s->F + ((long)k * N + n) * 3;
            double u[3], dU[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = (s->p.common_velocity && K > 1) ? ucommon[a] : jn[a] / r;
                dU[a] = Fn[a] / r;
            }
            double Cm[ORC_MAXQ];
            surface_source(s, n, k, Cm);
            collide_node(s, s->f + ((long)k * N + n) * Q, r, u, dU, k, Cm,
                         s->fpost + ((long)k * N + n) * Q);
        }
    }
}

/* (7) push streaming with halfway bounce-back (Eq. lbe_steps).
 * Each destination slot has exactly one writer, so the loop is race free. */
static void stream(orc_sim* s)
{
    long N = s->N;
    int Q = s->Q, K = s->p.ncomp;
    memset(s->fnew, 0, sizeof(double) * (size_t)(K * N * Q));
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->solid[n]) continue;
        int c[3];
        coords_of(s, n, c);
        for (int i = 0; i < Q; ++i) {
            long m = 0;
            int kind = stream_target(s, c, s->e[i], &m);
            for (int k = 0; k < K; ++k) {
                double v = s->fpost[((long)k * N + n) * Q + i];
                if (kind == 0) s->fnew[((long)k * N + m) * Q + i] = v;
                else if (kind == 1) s->fnew[((long)k * N + n) * Q + s->opp[i]] = v;
            }
        }
    }
}

/* (8) constant-density x faces: Zou-He closure with zero tangential velocity.
 * n_in = inward normal; unknown populations have e.n_in > 0:
 *   rho u_n = rho_b - (sum_{e.n=0} f + 2 sum_{e.n<0} f)
 *   f_i = f_opp(i) + 6 w_i rho_b u_n (e_i.n) - (1/2) e_i,t . N_t,
 *   N_t = sum_{e.n=0} f_j e_j,t  (t = components tangential to the face). */
static void pressure_faces_on(orc_sim* s, double* farr, int k0, int k1)
{
    int Q = s->Q;
    long N = s->N;
    for (int side = 0; side < 2; ++side) {
        if (s->p.face_bc[side] != ORC_PRESSURE) continue;
        int xface = side == 0 ? 0 : s->dims[0] - 1;
        int nin = side == 0 ? 1 : -1;
        for (int z = 0; z < s->dims[2]; ++z)
            for (int y = 0; y < s->dims[1]; ++y) {
                long n = node_of(s, xface, y, z);
                if (s->solid[n]) continue;
                for (int k = k0; k < k1; ++k) {
                    double* fn = farr + ((long)k * N + n) * Q;
                    double rb = s->p.face_rho[side][k];
                    double s0 = 0.0, sneg = 0.0, Nt[3] = {0, 0, 0};
                    for (int i = 0; i < Q; ++i) {
                        int en = s->e[i][0] * nin;
                        if (en == 0) {
                            s0 += fn[i];
                            Nt[1] += fn[i] * s->e[i][1];
                            Nt[2] += fn[i] * s->e[i][2];
                        } else if (en < 0) sneg += fn[i];
                    }
                    double run = rb - (s0 + 2.0 * sneg);
                    for (int i = 0; i < Q; ++i) {
                        int en = s->e[i][0] * nin;
                        if (en <= 0) continue;
                        double et = s->e[i][1] * Nt[1] + s->e[i][2] * Nt[2];
                        fn[i] = fn[s->opp[i]] + 6.0 * s->w[i] * run * en - 0.5 * et;
                    }
                }
            }
    }
}

static void pressure_faces(orc_sim* s) { pressure_faces_on(s, s->fnew, 0, s->p.ncomp); }

void orc_step(orc_sim* s, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        fields_and_force(s);
        collide(s);
        stream(s);
        pressure_faces(s);
        double* tmp = s->f; s->f = s->fnew; s->fnew = tmp;
        s->steps++;
    }
}

/* ------------------------------------------------------------------------ */
/* Outputs                                                                   */
/* ------------------------------------------------------------------------ */

/* Density and output velocity (sum_i f_i e_i + F/2) / rho at the current time.
 * k >= 0: component k; k < 0: mixture (sum over components). Solids give 0.
 * u is laid out [dim][N]. Either pointer may be NULL. */
void orc_macroscopic(orc_sim* s, int k, double* rho, double* u)
{
    fields_and_force(s);
    long N = s->N;
    int K = s->p.ncomp, d = s->p.dim;
    for (long n = 0; n < N; ++n) {
        double r = 0.0, m[3] = {0, 0, 0};
        if (!s->solid[n]) {
            for (int c = 0; c < K; ++c) {
                if (k >= 0 && c != k) continue;
                r += s->rho[(long)c * N + n];
                for (int a = 0; a < 3; ++a)
                    m[a] += s->j[((long)c * N + n) * 3 + a] + 0.5 * s->F[((long)c * N + n) * 3 + a];
            }
        }
        if (rho) rho[n] = r;
        if (u) for (int a = 0; a < d; ++a) u[(long)a * N + n] = r != 0.0 ? m[a] / r : 0.0;
    }
}

/* Force field at the current time (interaction + body), [dim][N] */
void orc_force(orc_sim* s, int k, double* F)
{
    fields_and_force(s);
    long N = s->N;
    for (long n = 0; n < N; ++n)
        for (int a = 0; a < s->p.dim; ++a) F[(long)a * N + n] = s->F[((long)k * N + n) * 3 + a];
}

/* psi field at the current time (fluid and boundary-solid nodes), [N] */
void orc_psi(orc_sim* s, int k, double* psi, double* rho_with_virtual)
{
    fields_and_force(s);
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (psi) psi[n] = s->psi[(long)k * N + n];
        if (rho_with_virtual) rho_with_virtual[n] = s->rho[(long)k * N + n];
    }
}

/* Total mass and momentum per component, summed in node order.
 * mom = sum (j + F/2) (physical momentum). mass[2], mom[2*3]. */
void orc_diagnostics(orc_sim* s, double* mass, double* mom)
{
    fields_and_force(s);
    long N = s->N;
    for (int k = 0; k < s->p.ncomp; ++k) {
        double m = 0.0, p[3] = {0, 0, 0};
        for (long n = 0; n < N; ++n) {
            if (s->solid[n]) continue;
            m += s->rho[(long)k * N + n];
            for (int a = 0; a < 3; ++a)
                p[a] += s->j[((long)k * N + n) * 3 + a] + 0.5 * s->F[((long)k * N + n) * 3 + a];
        }
        mass[k] = m;
        for (int a = 0; a < 3; ++a) mom[3 * k + a] = p[a];
    }
}

/* boundary-solid mask (solids read by the fluid stencils) */
void orc_boundary_solids(const orc_sim* s, uint8_t* out)
{
    memcpy(out, s->bsolid, (size_t)s->N);
}
