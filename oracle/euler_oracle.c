/*
 * Plain FP64 CPU oracle of the GP-WENO finite-difference scheme (FD-Prim) for
 * the compressible Euler equations.  TEST INFRASTRUCTURE ONLY: it is built and
 * called by tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py, never by the product path.  It shares no source with the CUDA
 * library.
 *
 * What it computes, per the paper:
 *   - conserved variables and fluxes of the Euler equations (Eq. euler), ideal
 *     gas p = (gamma-1)(E - rho|u|^2/2);
 *   - Riemann states U^L, U^R at every face by GP-WENO interpolation of the
 *     characteristic variables of the primitive variables (Section 3.2-3.3;
 *     Section 6 for the use of characteristic variables): candidate predictions q^m = w_m^T f_m
 *     (Eq. candidate_interp), smoothness indicators beta_m = f_m^T K_m^{-1} f_m
 *     (Eq. gp-smooth, the definition form), WENO-JS weights
 *     omega_m = gamma_m/(eps+beta_m)^p normalised (Eq. weights), combination
 *     q = sum omega_m q^m (Eq. weight_sum);
 *   - the face flux F_{i+1/2} = RP(U^L, U^R) (Eq. riemann_prob) taken as the
 *     local Lax-Friedrichs (Rusanov) flux, or the HLLC flux that the paper
 *     uses by default (Section 7);
 *   - the high-order correction f^ = F + alpha D^2F + beta D^4F with
 *     alpha = -1/24, beta = 3/640 on neighbouring face fluxes (Eqs. numFlux_cor,
 *     FD-ders);
 *   - the semi-discrete divergence (Eq. disc_fd) and the three-stage SSP-RK
 *     update in Shu-Osher form (Section 2, step 5).
 *
 * Readings where the paper is silent: the interpolated variables are the
 * characteristic variables of the primitive system (rho, u, p), "FD-Primitive"
 * (Section 1) with the projection of Section 6, using the eigenvectors of the
 * primitive-variable Jacobian at the Roe average of the two cells sharing the
 * face, in the basis written out in prim_eigensystem() below; local
 * Lax-Friedrichs speed max(|u_n|+c) over U^L and U^R; ghost cells by periodic
 * wrap or zero-gradient copy, G = R+3 layers (R+1 for the face stencil, two
 * more for the correction).
 *
 * Layout: U is structure-of-arrays [nc][nz][ny][nx], nc = ndim+2 components
 * (rho, rho u_1..rho u_ndim, E), interior cells only, FP64.
 *
 * Each quantity is computed once where it belongs: the primitive variables of
 * a cell once per RHS evaluation, the smoothness indicators of a window once
 * per face and field (with the zero-mean indicators the two states of a face
 * share R of their R+1 windows), the corrected flux once per face.
 *
 * Operation count.  Built with -DORACLE_COUNT_OPS, the OPS() annotations
 * tally the floating-point operations this file executes for the FD-Prim
 * scheme (the paper's algorithm in the order above): add, subtract,
 * multiply, divide and square root count one each, as does a max or min
 * that selects a value; sign changes, fabs, copies and validity checks count
 * nothing; a sum of k terms counts k-1 additions; pow(x, p) counts p-1
 * multiplications; terms of the eigenvector products whose coefficient is a
 * structural zero are skipped and a coefficient of +-1 costs no multiply.
 * oracle_ops() returns the tally (always 0 in the normal build, where OPS()
 * compiles to nothing).  The HLLC and HLL fluxes count the branch they take;
 * the FD-Flux and GP-AO paths are not annotated.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_COUNT_OPS
static unsigned long long g_ops = 0;
#define OPS(n) (g_ops += (unsigned long long)(n))
#else
#define OPS(n) ((void)0)
#endif

#define OR_MAXR 4
#define OR_MAXC 5
#define OR_MAXS (2 * OR_MAXR + 2)

typedef struct {
    int ndim;          /* 1, 2 or 3 */
    int n[3];          /* cells in x, y, z (unused dims = 1) */
    double dx[3];      /* grid spacing per dimension */
    int bc_lo[3];      /* 0 = periodic, 1 = outflow (zero gradient) */
    int bc_hi[3];
    int R;             /* GP radius, 1..4 */
    double gamma;      /* ratio of specific heats */
    double eps;        /* WENO epsilon (paper: 1e-36) */
    int p;             /* WENO power (paper: 2) */
    const double *wl;  /* [(R+1)][(R+1)] sub-stencil weights, prediction at x* = +1/2 */
    const double *gl;  /* [(R+1)] linear weights at x* = +1/2 */
    const double *wr;  /* [(R+1)][(R+1)] sub-stencil weights, prediction at x* = -1/2 */
    const double *gr;  /* [(R+1)] linear weights at x* = -1/2 */
    const double *Kinv;/* [(R+1)][(R+1)] inverse of K_m built with sigma */
    int flux;          /* 0 = local Lax-Friedrichs, 1 = HLLC, 2 = HLL */
    int beta_mean;     /* 0 = zero-mean GP smoothness indicators (the paper's choice), 1 = mean f_centre */
    int scheme;        /* 0 = FD-Prim (Riemann states + face flux + correction), 1 = FD-Flux (Section 2) */
    int ao;            /* 0 = GP-WENO; 1 = GP-AO (Appendix A): R = 2 gives AO(2,3), R = 3 gives AO(3,2,3) */
    double ao_gamma_hi, ao_gamma_lo;
    const double *ao_l;   /* x* = +1/2: w_hi[2R+1], w_lo[2R-1] (R = 3 only), w_3[3][3] */
    const double *ao_r;   /* the same at x* = -1/2 */
    const double *ao_kinv;/* K^-1 built with sigma: hi [(2R+1)^2], lo [(2R-1)^2] (R = 3 only), 3-point [9] */
    double ao_const[3];   /* constant terms added to beta of the hi, lo and 3-point stencils */
    double ao_scale[3];   /* factors of the data-fit terms of the hi, lo and 3-point stencils */
} oracle_cfg;

static long ncells(const oracle_cfg *c) { return (long)c->n[0] * c->n[1] * c->n[2]; }

/* Map a possibly out-of-range cell index along one dimension to the interior. */
static int map_index(const oracle_cfg *c, int d, int i)
{
    int n = c->n[d];
    if (i < 0) {
        if (c->bc_lo[d] == 0) { i %= n; if (i < 0) i += n; }
        else i = 0;
    } else if (i >= n) {
        if (c->bc_hi[d] == 0) i %= n;
        else i = n - 1;
    }
    return i;
}

static long lin(const oracle_cfg *c, int i, int j, int k)
{
    return ((long)k * c->n[1] + j) * c->n[0] + i;
}

/* Pressure of a conserved state (any number of dimensions). */
static double pressure(const double *u, int nc, double g)
{
    double ke = 0.0;
    for (int a = 1; a < nc - 1; ++a) ke += u[a] * u[a];
    OPS(2 * (nc - 2) - 1 + 5);
    return (g - 1.0) * (u[nc - 1] - 0.5 * ke / u[0]);
}

/* Physical flux in the direction whose momentum sits in slot 1 ("normal-first"
 * ordering).  Eq. euler. */
static void normal_flux(const double *u, int nc, double g, double *f)
{
    double rho = u[0], un = u[1] / rho, p = pressure(u, nc, g);
    f[0] = u[1];
    f[1] = u[1] * un + p;
    for (int a = 2; a < nc - 1; ++a) f[a] = u[a] * un;
    f[nc - 1] = un * (u[nc - 1] + p);
    OPS(1 + 2 + (nc - 3) + 2);
}

/* Roe average of two conserved states (normal-first ordering) with their
 * pressures pL, pR: density sqrt(rhoL rhoR), sqrt(rho)-weighted velocity and
 * total enthalpy, and the sound speed c^2 = (gamma-1)(H - |u|^2/2).
 * roe[0] = rho, roe[1..nv] = u, roe[nv+1] = H, roe[nv+2] = c.  Returns 0 if
 * c^2 <= 0 or a density <= 0. */
static int roe_average(const double *uL, const double *uR, double pL, double pR, int nc, double g, double *roe)
{
    int nv = nc - 2;
    if (!(uL[0] > 0.0) || !(uR[0] > 0.0)) return 0;
    double sL = sqrt(uL[0]), sR = sqrt(uR[0]);
    double HL = (uL[nc - 1] + pL) / uL[0], HR = (uR[nc - 1] + pR) / uR[0];
    double q2 = 0.0;
    roe[0] = sL * sR;
    for (int a = 0; a < nv; ++a) {
        roe[1 + a] = (sL * uL[1 + a] / uL[0] + sR * uR[1 + a] / uR[0]) / (sL + sR);
        q2 += roe[1 + a] * roe[1 + a];
    }
    double H = (sL * HL + sR * HR) / (sL + sR);
    double c2 = (g - 1.0) * (H - 0.5 * q2);
    OPS(2 + 4 + 1 + 9 * nv - 1 + 5 + 4 + 1);
    roe[nv + 1] = H;
    if (!(c2 > 0.0)) return 0;
    roe[nv + 2] = sqrt(c2);
    return 1;
}

/* Right (columns of Rm) and left (rows of Lm) eigenvectors of the
 * primitive-variable Euler system V_t + A_V V_x = 0, V = (rho, u_n,
 * u_t..., p) normal-first, at density rho and sound speed c (taken from the
 * Roe average of the two cells sharing the face).  Waves in the order
 * u-c, entropy, one shear wave per tangential velocity, u+c:
 *   L rows: (0, -rho/(2c), 0, 1/(2c^2)), (1, 0, 0, -1/c^2), e_t, (0, rho/(2c), 0, 1/(2c^2))
 *   R cols: (1, -c/rho, 0, c^2),         (1, 0, 0, 0),      e_t, (1, c/rho, 0, c^2). */
static void prim_eigensystem(double rho, double c, int nc, double Rm[OR_MAXC][OR_MAXC], double Lm[OR_MAXC][OR_MAXC])
{
    int E = nc - 1;
    double an = rho / (2.0 * c), c2 = c * c, ap = 1.0 / (2.0 * c2), ie = 1.0 / c2, cr = c / rho;
    OPS(7);
    memset(Rm, 0, sizeof(double) * OR_MAXC * OR_MAXC);
    memset(Lm, 0, sizeof(double) * OR_MAXC * OR_MAXC);
    Lm[0][1] = -an;
    Lm[0][E] = ap;
    Lm[1][0] = 1.0;
    Lm[1][E] = -ie;
    for (int t = 2; t < E; ++t) Lm[t][t] = 1.0;
    Lm[E][1] = an;
    Lm[E][E] = ap;
    Rm[0][0] = 1.0;
    Rm[1][0] = -cr;
    Rm[E][0] = c2;
    Rm[0][1] = 1.0;
    for (int t = 2; t < E; ++t) Rm[t][t] = 1.0;
    Rm[0][E] = 1.0;
    Rm[1][E] = cr;
    Rm[E][E] = c2;
}

/* row . v over the non-zero entries of a row of an eigenvector matrix (the
 * zeros are structural; a coefficient of +-1 needs no multiply). */
static double dot_sparse(const double *row, const double *v, int n)
{
    double acc = 0.0;
    int first = 1;
    for (int a = 0; a < n; ++a) {
        if (row[a] == 0.0) continue;
        acc += row[a] * v[a];
        OPS((fabs(row[a]) == 1.0 ? 0 : 1) + (first ? 0 : 1));
        first = 0;
    }
    (void)first;
    return acc;
}

/* Primitive variables (rho, u..., p) of a conserved state, same ordering. */
static void to_primitive(const double *u, int nc, double g, double *v)
{
    v[0] = u[0];
    for (int a = 1; a < nc - 1; ++a) v[a] = u[a] / u[0];
    OPS(nc - 2);
    v[nc - 1] = pressure(u, nc, g);
}

static void to_conserved(const double *v, int nc, double g, double *u)
{
    double ke = 0.0;
    u[0] = v[0];
    for (int a = 1; a < nc - 1; ++a) {
        u[a] = v[0] * v[a];
        ke += v[a] * v[a];
    }
    u[nc - 1] = v[nc - 1] / (g - 1.0) + 0.5 * v[0] * ke;
    OPS(3 * (nc - 2) - 1 + 5);
}

/* GP smoothness indicator of one sub-stencil window f[0..R] (Eq. gp-smooth):
 * beta = d^T K^-1 d with d = f - mean, evaluated as d . (K^-1 d); mean = 0 for
 * the zero-mean GP, the centre value f_i of the stencil with a non-zero mean
 * (Section 3.3, the variant of Section 7.1). */
static double beta_window(const oracle_cfg *c, const double *f, double mean)
{
    int S = c->R + 1;
    double d[OR_MAXR + 1], beta = 0.0;
    for (int a = 0; a < S; ++a) d[a] = c->beta_mean ? f[a] - mean : f[a];
    if (c->beta_mean) OPS(S);
    for (int a = 0; a < S; ++a) {
        double y = 0.0;
        for (int b = 0; b < S; ++b) y += c->Kinv[a * S + b] * d[b];
        beta += d[a] * y;
    }
    OPS(S * (2 * S - 1) + 2 * S - 1);
    return beta;
}

/* Smoothness indicators of the sub-stencils of both states of a face from the
 * 2R+2 values f[0..2R+1] (cells s-R .. s+1+R): bl[m] of window f[m..m+R]
 * (left state, stencil of cell s) and br[m] of window f[1+m..1+m+R] (right
 * state, stencil of cell s+1).  With the zero mean the windows shared by the
 * two states are evaluated once. */
static void face_betas(const oracle_cfg *c, const double *f, double *bl, double *br)
{
    int R = c->R;
    if (!c->beta_mean) {
        double b[OR_MAXR + 2];
        for (int w = 0; w <= R + 1; ++w) b[w] = beta_window(c, f + w, 0.0);
        for (int m = 0; m <= R; ++m) {
            bl[m] = b[m];
            br[m] = b[m + 1];
        }
        return;
    }
    for (int m = 0; m <= R; ++m) {
        bl[m] = beta_window(c, f + m, f[R]);
        br[m] = beta_window(c, f + 1 + m, f[R + 1]);
    }
}

/* GP-WENO prediction at one face centre from 2R+1 values f[0..2R] centred on
 * the cell whose stencil is used and the smoothness indicators beta[m] of its
 * sub-stencils; w: (R+1)x(R+1) sub-stencil weights, gam: linear weights.
 * Sub-stencil m covers f[m..m+R] (Eq. sub-stencil). */
static double gp_weno(const oracle_cfg *c, const double *f, const double *w, const double *gam,
                      const double *beta)
{
    int R = c->R, S = R + 1;
    double q[OR_MAXR + 1], wt[OR_MAXR + 1], wsum = 0.0, out = 0.0;
    for (int m = 0; m < S; ++m) {
        const double *fm = f + m;
        double qm = 0.0;
        for (int j = 0; j < S; ++j) qm += w[m * S + j] * fm[j];              /* Eq. candidate_interp */
        q[m] = qm;
        wt[m] = gam[m] / pow(c->eps + beta[m], (double)c->p);                  /* Eq. weights */
        wsum += wt[m];
    }
    for (int m = 0; m < S; ++m) out += (wt[m] / wsum) * q[m];                   /* Eq. weight_sum */
    OPS(S * (2 * S - 1) + S * (2 + (c->p - 1)) + (S - 1) + 3 * S - 1);
    return out;
}

/* beta of one stencil for GP-AO: the data-fit term of the negative log-likelihood,
 * (1/2) f^T K^-1 f (Eq. log-like; f relative to the centre value with beta_mean),
 * plus the configured constant (the normalisation and complexity terms). */
static double ao_beta(const oracle_cfg *c, const double *Kinv, const double *f, int n, double mean, double cst,
                      double scale)
{
    double b = 0.0;
    for (int a = 0; a < n; ++a)
        for (int d = 0; d < n; ++d) b += (f[a] - mean) * Kinv[a * n + d] * (f[d] - mean);
    return scale * 0.5 * b + cst;
}

/* GP-AO(R,3) (Eq. GP-AO): the high-order prediction qh with its beta bh hybridised with the
 * three 3-point predictions q3 and betas b3.  Nonlinear weights Eq. nonlin-AO with
 * gamma_HI for the high-order stencil and gamma_m (Eq. CWENO-lin) for the small ones. */
static double ao_r3(const oracle_cfg *c, double qh, double bh, const double *q3, const double *b3)
{
    double ghi = c->ao_gamma_hi, glo = c->ao_gamma_lo;
    double g[3] = { 0.5 * (1.0 - ghi) * (1.0 - glo), (1.0 - ghi) * glo, 0.5 * (1.0 - ghi) * (1.0 - glo) };
    double wh = ghi / pow(c->eps + bh, (double)c->p), w[3], sum = wh;
    for (int m = 0; m < 3; ++m) {
        w[m] = g[m] / pow(c->eps + b3[m], (double)c->p);
        sum += w[m];
    }
    double oh = wh / sum;
    double q = oh / ghi * qh;
    for (int m = 0; m < 3; ++m) q += (w[m] / sum - oh / ghi * g[m]) * q3[m];
    return q;
}

/* GP-AO prediction at one face centre from the 2R+1 values f[0..2R] centred on the
 * stencil's cell (Appendix A): R = 2 gives AO(2,3); R = 3 gives the recursive
 * AO(3,2,3) of Eqs. recursive-weights and AO-recursive. */
static double gp_ao(const oracle_cfg *c, const double *f, const double *tab)
{
    int R = c->R, nh = 2 * R + 1, nl = R == 3 ? 2 * R - 1 : 0;
    const double *w_hi = tab, *w_lo = tab + nh, *w3 = w_lo + nl;
    const double *K_hi = c->ao_kinv, *K_lo = K_hi + nh * nh, *K3 = K_lo + nl * nl;
    double mean = c->beta_mean ? f[R] : 0.0;
    double q3[3], b3[3];
    for (int m = 0; m < 3; ++m) {
        const double *fm = f + R - 2 + m;     /* Eq. cweno_stencil: cells i-2..i, i-1..i+1, i..i+2 */
        q3[m] = 0.0;
        for (int j = 0; j < 3; ++j) q3[m] += w3[m * 3 + j] * fm[j];
        b3[m] = ao_beta(c, K3, fm, 3, mean, c->ao_const[2], c->ao_scale[2]);
    }
    double qh = 0.0;
    for (int j = 0; j < nh; ++j) qh += w_hi[j] * f[j];
    double bh = ao_beta(c, K_hi, f, nh, mean, c->ao_const[0], c->ao_scale[0]);
    double q_hi = ao_r3(c, qh, bh, q3, b3);
    if (R == 2) return q_hi;
    double ql = 0.0;
    for (int j = 0; j < nl; ++j) ql += w_lo[j] * f[1 + j];
    double bl = ao_beta(c, K_lo, f + 1, nl, mean, c->ao_const[1], c->ao_scale[1]);
    double q_lo = ao_r3(c, ql, bl, q3, b3);
    double ghi = c->ao_gamma_hi;
    double vh = ghi / pow(c->eps + bh, (double)c->p), vl = (1.0 - ghi) / pow(c->eps + bl, (double)c->p);
    double nuh = vh / (vh + vl), nul = vl / (vh + vl);
    return nuh / ghi * q_hi + (nul - nuh / ghi * (1.0 - ghi)) * q_lo;
}

/* HLLC flux (Toro's three-wave approximate Riemann solver) of two conserved
 * normal-first states, with the wave speeds of Einfeldt from the Roe average:
 * S_L = min(u_L - c_L, u_roe - c_roe), S_R = max(u_R + c_R, u_roe + c_roe),
 * contact speed S* from the momentum jump, star states
 * U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S*, v_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))). */
static void hllc_flux(const double *uL, const double *uR, int nc, double g, double uroe, double croe, double *F)
{
    int E = nc - 1;
    double rL = uL[0], rR = uR[0];
    double vL = uL[1] / rL, vR = uR[1] / rR;
    double pL = pressure(uL, nc, g), pR = pressure(uR, nc, g);
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double SL = fmin(vL - cL, uroe - croe), SR = fmax(vR + cR, uroe + croe);
    double Ss = (pR - pL + rL * vL * (SL - vL) - rR * vR * (SR - vR)) / (rL * (SL - vL) - rR * (SR - vR));
    double fL[OR_MAXC], fR[OR_MAXC];
    normal_flux(uL, nc, g, fL);
    normal_flux(uR, nc, g, fR);
    OPS(2 + 6 + 6 + 15);
    if (SL >= 0.0) {
        for (int a = 0; a < nc; ++a) F[a] = fL[a];
        return;
    }
    if (SR <= 0.0) {
        for (int a = 0; a < nc; ++a) F[a] = fR[a];
        return;
    }
    const double *uK = Ss >= 0.0 ? uL : uR;
    const double *fK = Ss >= 0.0 ? fL : fR;
    double rK = uK[0], vK = uK[1] / rK, pK = Ss >= 0.0 ? pL : pR, SK = Ss >= 0.0 ? SL : SR;
    double chi = rK * (SK - vK) / (SK - Ss);
    double us[OR_MAXC];
    us[0] = chi;
    us[1] = chi * Ss;
    for (int a = 2; a < E; ++a) us[a] = chi * uK[a] / rK;
    us[E] = chi * (uK[E] / rK + (Ss - vK) * (Ss + pK / (rK * (SK - vK))));
    for (int a = 0; a < nc; ++a) F[a] = fK[a] + SK * (us[a] - uK[a]);
    OPS(1 + 4 + 1 + 2 * (nc - 3) + 9 + 3 * nc);
}

/* HLL flux (Harten, Lax and van Leer's two-wave solver) of two conserved
 * normal-first states with the same Einfeldt speeds as hllc_flux:
 * F = F_L if S_L >= 0, F_R if S_R <= 0, else
 * (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L). */
static void hll_flux(const double *uL, const double *uR, int nc, double g, double uroe, double croe, double *F)
{
    double rL = uL[0], rR = uR[0];
    double vL = uL[1] / rL, vR = uR[1] / rR;
    double pL = pressure(uL, nc, g), pR = pressure(uR, nc, g);
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double SL = fmin(vL - cL, uroe - croe), SR = fmax(vR + cR, uroe + croe);
    double fL[OR_MAXC], fR[OR_MAXC];
    normal_flux(uL, nc, g, fL);
    normal_flux(uR, nc, g, fR);
    OPS(2 + 6 + 6);
    for (int a = 0; a < nc; ++a) {
        if (SL >= 0.0) F[a] = fL[a];
        else if (SR <= 0.0) F[a] = fR[a];
        else {
            F[a] = (SR * fL[a] - SL * fR[a] + SL * SR * (uR[a] - uL[a])) / (SR - SL);
            OPS(9);
        }
    }
}

/* The 2R+2 cells s-R .. s+1+R along dimension d at transverse position cell,
 * in normal-first component order (perm maps normal-first -> natural). */
static void gather_stencil(const oracle_cfg *c, const double *U, int d, int s, const int cell[3], int perm[OR_MAXC],
                           double st[OR_MAXS][OR_MAXC])
{
    int nc = c->ndim + 2, R = c->R, ns = 2 * R + 2;
    long N = ncells(c);
    perm[0] = 0; perm[1] = 1 + d;
    int k = 2;
    for (int a = 0; a < c->ndim; ++a) if (a != d) perm[k++] = 1 + a;
    perm[nc - 1] = nc - 1;
    for (int q = 0; q < ns; ++q) {
        int idx[3] = { cell[0], cell[1], cell[2] };
        idx[d] = map_index(c, d, s - R + q);
        long l = lin(c, idx[0], idx[1], idx[2]);
        for (int a = 0; a < nc; ++a) st[q][a] = U[(long)perm[a] * N + l];
    }
}

/* Primitive variables of the same stencil (from the primitive array V of the
 * whole grid, same layout as U). */
static void gather_prim(const oracle_cfg *c, const double *V, int d, int s, const int cell[3], const int perm[OR_MAXC],
                        double vs[OR_MAXS][OR_MAXC])
{
    int nc = c->ndim + 2, R = c->R, ns = 2 * R + 2;
    long N = ncells(c);
    for (int q = 0; q < ns; ++q) {
        int idx[3] = { cell[0], cell[1], cell[2] };
        idx[d] = map_index(c, d, s - R + q);
        long l = lin(c, idx[0], idx[1], idx[2]);
        for (int a = 0; a < nc; ++a) vs[q][a] = V[(long)perm[a] * N + l];
    }
}

/* Normal flux of a state from its primitive (v) and conserved (u) forms,
 * normal-first ordering (Eq. euler). */
static void flux_prim(const double *v, const double *u, int nc, double *f)
{
    double un = v[1], p = v[nc - 1];
    f[0] = u[1];
    f[1] = u[1] * un + p;
    for (int a = 2; a < nc - 1; ++a) f[a] = u[a] * un;
    f[nc - 1] = un * (u[nc - 1] + p);
    OPS(2 + (nc - 3) + 2);
}

/* Face flux F between stencil cells R and R+1 of the conserved stencil st and
 * its primitive variables vs (2R+2 cells, normal-first).  Writes nc values
 * (normal-first order) and, if asked, the Riemann states.  Returns 0 on a
 * non-physical state. */
static int face_flux(const oracle_cfg *c, double st[OR_MAXS][OR_MAXC], double vs[OR_MAXS][OR_MAXC], double *Fn,
                     double *uLout, double *uRout)
{
    int nc = c->ndim + 2, R = c->R, ns = 2 * R + 2;
    double roe[OR_MAXC + 1];
    if (!roe_average(st[R], st[R + 1], vs[R][nc - 1], vs[R + 1][nc - 1], nc, c->gamma, roe)) return 0;
    double Rm[OR_MAXC][OR_MAXC], Lm[OR_MAXC][OR_MAXC];
    prim_eigensystem(roe[0], roe[nc], nc, Rm, Lm);

    /* characteristic projection of the primitive variables of every stencil cell */
    double ch[OR_MAXC][OR_MAXS];
    for (int q = 0; q < ns; ++q)
        for (int f = 0; f < nc; ++f) ch[f][q] = dot_sparse(Lm[f], vs[q], nc);
    double wL[OR_MAXC], wR[OR_MAXC];
    for (int f = 0; f < nc; ++f) {
        /* cells s-R..s+R at x* = +1/2; cells s+1-R..s+1+R at x* = -1/2 */
        if (c->ao) {
            wL[f] = gp_ao(c, &ch[f][0], c->ao_l);
            wR[f] = gp_ao(c, &ch[f][1], c->ao_r);
        } else {
            double bl[OR_MAXR + 1], br[OR_MAXR + 1];
            face_betas(c, ch[f], bl, br);
            wL[f] = gp_weno(c, &ch[f][0], c->wl, c->gl, bl);
            wR[f] = gp_weno(c, &ch[f][1], c->wr, c->gr, br);
        }
    }
    /* back to primitive states with the right eigenvectors */
    double vL[OR_MAXC], vR[OR_MAXC], uL[OR_MAXC], uR[OR_MAXC];
    for (int a = 0; a < nc; ++a) {
        vL[a] = dot_sparse(Rm[a], wL, nc);
        vR[a] = dot_sparse(Rm[a], wR, nc);
    }
    if (!(vL[0] > 0.0) || !(vR[0] > 0.0) || !(vL[nc - 1] > 0.0) || !(vR[nc - 1] > 0.0)) return 0;
    to_conserved(vL, nc, c->gamma, uL);
    to_conserved(vR, nc, c->gamma, uR);
    if (c->flux == 1) {
        hllc_flux(uL, uR, nc, c->gamma, roe[1], roe[nc], Fn);
    } else if (c->flux == 2) {
        hll_flux(uL, uR, nc, c->gamma, roe[1], roe[nc], Fn);
    } else {
        /* local Lax-Friedrichs: alpha = max(|u_n| + c) over the two states */
        double cL = sqrt(c->gamma * vL[nc - 1] / vL[0]), cR = sqrt(c->gamma * vR[nc - 1] / vR[0]);
        double aL = fabs(vL[1]) + cL, aR = fabs(vR[1]) + cR;
        double alpha = aL > aR ? aL : aR;
        double ha = 0.5 * alpha;
        double fL[OR_MAXC], fR[OR_MAXC];
        flux_prim(vL, uL, nc, fL);
        flux_prim(vR, uR, nc, fR);
        for (int a = 0; a < nc; ++a) Fn[a] = 0.5 * (fL[a] + fR[a]) - ha * (uR[a] - uL[a]);
        OPS(2 * 4 + 1 + 1 + 5 * nc);
    }
    if (uLout) memcpy(uLout, uL, sizeof(double) * nc);
    if (uRout) memcpy(uRout, uR, sizeof(double) * nc);
    return 1;
}

/* Right eigenvectors (columns of Rc) of the conservative normal-flux Jacobian
 * dF/dU at velocity vel (normal first), total enthalpy H and sound speed c,
 * waves in the order u-c, entropy, one shear wave per tangential velocity,
 * u+c (textbook form):
 *   (1, u - c e_n, H - u_n c), (1, u, |u|^2/2), (0, e_t, u_t), (1, u + c e_n, H + u_n c);
 * the left eigenvectors Lc = Rc^{-1} by Gauss-Jordan elimination with partial
 * pivoting.  Returns 0 if Rc is singular. */
static int cons_eigensystem(const double *vel, double H, double c, int nc, double Rc[OR_MAXC][OR_MAXC],
                            double Lc[OR_MAXC][OR_MAXC])
{
    int E = nc - 1, nv = nc - 2;
    double q2 = 0.0;
    for (int a = 0; a < nv; ++a) q2 += vel[a] * vel[a];
    memset(Rc, 0, sizeof(double) * OR_MAXC * OR_MAXC);
    Rc[0][0] = 1.0;
    Rc[0][1] = 1.0;
    Rc[0][E] = 1.0;
    for (int a = 0; a < nv; ++a) {
        Rc[1 + a][0] = vel[a] - (a == 0 ? c : 0.0);
        Rc[1 + a][1] = vel[a];
        Rc[1 + a][E] = vel[a] + (a == 0 ? c : 0.0);
    }
    Rc[E][0] = H - vel[0] * c;
    Rc[E][1] = 0.5 * q2;
    Rc[E][E] = H + vel[0] * c;
    for (int t = 1; t < nv; ++t) {
        Rc[1 + t][1 + t] = 1.0;
        Rc[E][1 + t] = vel[t];
    }
    double A[OR_MAXC][2 * OR_MAXC];
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < 2 * nc; ++j) A[i][j] = j < nc ? Rc[i][j] : (j - nc == i ? 1.0 : 0.0);
    for (int col = 0; col < nc; ++col) {
        int piv = col;
        for (int r = col + 1; r < nc; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return 0;
        for (int j = 0; j < 2 * nc; ++j) {
            double t = A[col][j];
            A[col][j] = A[piv][j];
            A[piv][j] = t;
        }
        double inv = 1.0 / A[col][col];
        for (int j = 0; j < 2 * nc; ++j) A[col][j] *= inv;
        for (int r = 0; r < nc; ++r) {
            if (r == col || A[r][col] == 0.0) continue;
            double f = A[r][col];
            for (int j = 0; j < 2 * nc; ++j) A[r][j] -= f * A[col][j];
        }
    }
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j) Lc[i][j] = A[i][nc + j];
    return 1;
}

/* FD-Flux numerical flux at face s+1/2 (Section 2): the point fluxes F_j are
 * read as cell averages of the function whose face value is the numerical
 * flux (Eqs. prim_F, design), split by local Lax-Friedrichs into parts
 * moving right and left, F^+- = (F +- alpha U)/2 with alpha = max over the
 * 2R+2 stencil cells of |u_n| + c, projected on the characteristic fields
 * of the conservative Jacobian at the Roe average of cells s and s+1, and
 * reconstructed by GP-WENO: F^+ from the stencil of cell s at x* = +1/2,
 * F^- from the stencil of cell s+1 at x* = -1/2 (the tables hold
 * reconstruction weights).  Returns 0 on a non-physical state. */
static int face_flux_fd(const oracle_cfg *c, const double *U, int d, int s, const int cell[3], double *Fout)
{
    int nc = c->ndim + 2, R = c->R, ns = 2 * R + 2;
    int perm[OR_MAXC];
    double st[OR_MAXS][OR_MAXC];
    gather_stencil(c, U, d, s, cell, perm, st);
    double roe[OR_MAXC + 1];
    if (!roe_average(st[R], st[R + 1], pressure(st[R], nc, c->gamma), pressure(st[R + 1], nc, c->gamma), nc,
                     c->gamma, roe))
        return 0;
    double Rc[OR_MAXC][OR_MAXC], Lc[OR_MAXC][OR_MAXC];
    if (!cons_eigensystem(&roe[1], roe[nc - 1], roe[nc], nc, Rc, Lc)) return 0;
    double alpha = 0.0;
    for (int q = 0; q < ns; ++q) {
        double p = pressure(st[q], nc, c->gamma);
        if (!(st[q][0] > 0.0) || !(p > 0.0)) return 0;
        double a = fabs(st[q][1] / st[q][0]) + sqrt(c->gamma * p / st[q][0]);
        if (a > alpha) alpha = a;
    }
    double gp[OR_MAXC][OR_MAXS], gm[OR_MAXC][OR_MAXS];
    for (int q = 0; q < ns; ++q) {
        double F[OR_MAXC];
        normal_flux(st[q], nc, c->gamma, F);
        for (int f = 0; f < nc; ++f) {
            double v = 0.0, g = 0.0;
            for (int a = 0; a < nc; ++a) {
                v += Lc[f][a] * st[q][a];
                g += Lc[f][a] * F[a];
            }
            gp[f][q] = 0.5 * (g + alpha * v);
            gm[f][q] = 0.5 * (g - alpha * v);
        }
    }
    double hat[OR_MAXC];
    for (int f = 0; f < nc; ++f) {
        if (c->ao) {
            hat[f] = gp_ao(c, &gp[f][0], c->ao_l) + gp_ao(c, &gm[f][1], c->ao_r);
            continue;
        }
        /* the two split parts have separate data, hence separate windows */
        double bl[OR_MAXR + 1], br[OR_MAXR + 1];
        for (int m = 0; m <= R; ++m) {
            bl[m] = beta_window(c, &gp[f][m], gp[f][R]);
            br[m] = beta_window(c, &gm[f][1 + m], gm[f][R + 1]);
        }
        hat[f] = gp_weno(c, &gp[f][0], c->wl, c->gl, bl) + gp_weno(c, &gm[f][1], c->wr, c->gr, br);
    }
    for (int a = 0; a < nc; ++a) {
        double acc = 0.0;
        for (int f = 0; f < nc; ++f) acc += Rc[a][f] * hat[f];
        Fout[perm[a]] = acc;
    }
    return 1;
}

/* Corrected numerical flux at face s+1/2 from the five face fluxes
 * F_{s-3/2} .. F_{s+5/2} (Eqs. numFlux_cor and FD-ders, alpha = -1/24,
 * beta = 3/640; the Delta^2 and Delta^4 factors cancel). */
static double corrected_flux(const double *F5)
{
    const double A2 = -1.0 / 24.0, A4 = 3.0 / 640.0;
    double D2 = F5[1] - 2.0 * F5[2] + F5[3];
    double D4 = F5[0] - 4.0 * F5[1] + 6.0 * F5[2] - 4.0 * F5[3] + F5[4];
    OPS(3 + 7 + 4);
    return F5[2] + A2 * D2 + A4 * D4;
}

double oracle_corrected_flux(const double *F5) { return corrected_flux(F5); }

/* dUdt = L(U), Eq. disc_fd with the corrected fluxes of Eq. numFlux_cor.
 * Per direction and grid line: the face fluxes F_{s+1/2}, s = -3 .. n+1, then
 * the corrected flux of each face s = -1 .. n-1 once, then the differences.
 * Returns 0 on success, 1 if any non-physical state was met. */
int oracle_rhs(const oracle_cfg *c, const double *U, double *dUdt)
{
    int nc = c->ndim + 2;
    long N = ncells(c);
    int bad = 0;
    memset(dUdt, 0, sizeof(double) * nc * N);
    /* FD-Prim: the primitive variables of every cell, once per evaluation */
    double *V = NULL;
    if (c->scheme == 0) {
        V = (double *)malloc(sizeof(double) * nc * N);
        for (long l = 0; l < N; ++l) {
            double u[OR_MAXC], v[OR_MAXC];
            for (int a = 0; a < nc; ++a) u[a] = U[(long)a * N + l];
            to_primitive(u, nc, c->gamma, v);
            for (int a = 0; a < nc; ++a) V[(long)a * N + l] = v[a];
        }
    }
    for (int d = 0; d < c->ndim; ++d) {
        int n = c->n[d];
        int nf = n + 5;                     /* faces s = -3 .. n+1 */
        double *F = (double *)malloc(sizeof(double) * nf * nc);
        double *Fh = (double *)malloc(sizeof(double) * (n + 1) * nc);   /* corrected, faces s = -1 .. n-1 */
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int b = 0; b < c->n[t2]; ++b)
            for (int a = 0; a < c->n[t1]; ++a) {
                int cell[3];
                cell[t1] = a; cell[t2] = b; cell[d] = 0;
                for (int s = -3; s <= n + 1; ++s) {
                    double *Fs = &F[(s + 3) * nc];
                    int ok;
                    if (c->scheme == 1) {
                        ok = face_flux_fd(c, U, d, s, cell, Fs);
                    } else {
                        int perm[OR_MAXC];
                        double st[OR_MAXS][OR_MAXC], vs[OR_MAXS][OR_MAXC], Fn[OR_MAXC];
                        gather_stencil(c, U, d, s, cell, perm, st);
                        gather_prim(c, V, d, s, cell, perm, vs);
                        ok = face_flux(c, st, vs, Fn, NULL, NULL);
                        for (int q = 0; q < nc; ++q) Fs[perm[q]] = Fn[q];
                    }
                    if (!ok) {
                        bad = 1;
                        for (int q = 0; q < nc; ++q) Fs[q] = NAN;
                    }
                }
                for (int t = -1; t <= n - 1; ++t)
                    for (int q = 0; q < nc; ++q) {
                        double F5[5];   /* faces t-2 .. t+2; F index of face s is s+3 */
                        for (int e = 0; e < 5; ++e) F5[e] = F[(t + 1 + e) * nc + q];
                        /* FD-Flux: the reconstructed flux is the numerical flux (Eq. design) */
                        Fh[(t + 1) * nc + q] = c->scheme == 1 ? F5[2] : corrected_flux(F5);
                    }
                for (int i = 0; i < n; ++i) {
                    cell[d] = i;
                    long l = lin(c, cell[0], cell[1], cell[2]);
                    for (int q = 0; q < nc; ++q)
                        dUdt[(long)q * N + l] -= (Fh[(i + 1) * nc + q] - Fh[i * nc + q]) / c->dx[d];
                    OPS(3 * nc);
                }
            }
        free(F);
        free(Fh);
    }
    free(V);
    return bad;
}

/* One SSP-RK3 step, Shu-Osher form:
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U = 1/3 U + 2/3 (U2 + dt L(U2)). */
int oracle_rk3_step(const oracle_cfg *c, double *U, double dt)
{
    int nc = c->ndim + 2;
    long M = (long)nc * ncells(c);
    double *L = (double *)malloc(sizeof(double) * M);
    double *U1 = (double *)malloc(sizeof(double) * M);
    double *U2 = (double *)malloc(sizeof(double) * M);
    int bad = 0;
    bad |= oracle_rhs(c, U, L);
    for (long i = 0; i < M; ++i) U1[i] = U[i] + dt * L[i];
    bad |= oracle_rhs(c, U1, L);
    for (long i = 0; i < M; ++i) U2[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * L[i]);
    bad |= oracle_rhs(c, U2, L);
    for (long i = 0; i < M; ++i) U[i] = U[i] / 3.0 + 2.0 / 3.0 * (U2[i] + dt * L[i]);
    OPS(M * (2 + 5 + 5));
    free(L); free(U1); free(U2);
    return bad;
}

/* Maximum of (|u_d| + c)/dx_d per dimension d; sum over d.  dt = cfl / result. */
double oracle_max_rate(const oracle_cfg *c, const double *U)
{
    int nc = c->ndim + 2;
    long N = ncells(c);
    double tot = 0.0;
    for (int d = 0; d < c->ndim; ++d) {
        double mx = 0.0;
        for (long l = 0; l < N; ++l) {
            double u[OR_MAXC];
            for (int a = 0; a < nc; ++a) u[a] = U[(long)a * N + l];
            double p = pressure(u, nc, c->gamma);
            double s = fabs(u[1 + d] / u[0]) + sqrt(c->gamma * p / u[0]);
            if (s > mx) mx = s;
        }
        tot += mx / c->dx[d];
    }
    return tot;
}

/* HLLC flux of two conserved normal-first states with given Roe velocity and
 * sound speed, exposed for unit tests. */
void oracle_hllc(int nc, double g, const double *uL, const double *uR, double uroe, double croe, double *F)
{
    hllc_flux(uL, uR, nc, g, uroe, croe, F);
}

/* HLL flux, exposed for unit tests (arguments as oracle_hllc). */
void oracle_hll(int nc, double g, const double *uL, const double *uR, double uroe, double croe, double *F)
{
    hll_flux(uL, uR, nc, g, uroe, croe, F);
}

/* Single face, exposed for unit tests: Riemann states and flux at the face
 * between stencil cells R and R+1 of a 1D stencil st[2R+2][nc] given in
 * natural order with the normal direction d.  Outputs uL, uR, F (nc each). */
int oracle_face(const oracle_cfg *c, int d, const double *st, double *uL, double *uR, double *F)
{
    /* Build a scratch grid of 2R+2 cells along d (others = 1) and gather the
     * stencil from it as oracle_rhs does, so the unit test exercises the same code. */
    oracle_cfg g = *c;
    int ns = 2 * c->R + 2, nc = c->ndim + 2;
    for (int a = 0; a < 3; ++a) { g.n[a] = 1; g.bc_lo[a] = g.bc_hi[a] = 1; }
    g.n[d] = ns;
    double *U = (double *)malloc(sizeof(double) * ns * nc);
    for (int q = 0; q < ns; ++q)
        for (int a = 0; a < nc; ++a) U[(long)a * ns + q] = st[q * nc + a];
    int cell[3] = { 0, 0, 0 }, perm[OR_MAXC];
    double gs[OR_MAXS][OR_MAXC], vs[OR_MAXS][OR_MAXC], Fn[OR_MAXC], uLn[OR_MAXC], uRn[OR_MAXC];
    gather_stencil(&g, U, d, c->R, cell, perm, gs);
    for (int q = 0; q < ns; ++q) to_primitive(gs[q], nc, c->gamma, vs[q]);
    int ok = face_flux(&g, gs, vs, Fn, uLn, uRn);
    if (ok)
        for (int a = 0; a < nc; ++a) {
            F[perm[a]] = Fn[a];
            uL[perm[a]] = uLn[a];
            uR[perm[a]] = uRn[a];
        }
    free(U);
    return ok;
}

/* Roe average (rho, u..., H, c) of two conserved states and the primitive
 * eigen-system at it (normal-first ordering), exposed for unit tests. */
int oracle_roe(int nc, double g, const double *uL, const double *uR, double *roe, double *Rout, double *Lout)
{
    double Rm[OR_MAXC][OR_MAXC], Lm[OR_MAXC][OR_MAXC];
    if (!roe_average(uL, uR, pressure(uL, nc, g), pressure(uR, nc, g), nc, g, roe)) return 0;
    prim_eigensystem(roe[0], roe[nc], nc, Rm, Lm);
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) { Rout[a * nc + b] = Rm[a][b]; Lout[a * nc + b] = Lm[a][b]; }
    return 1;
}

/* GP-WENO prediction exposed for unit tests: f has 2R+1 values. */
double oracle_gp_weno(const oracle_cfg *c, const double *f, int right)
{
    if (c->ao) return gp_ao(c, f, right ? c->ao_r : c->ao_l);
    double beta[OR_MAXR + 1];
    for (int m = 0; m <= c->R; ++m) beta[m] = beta_window(c, f + m, f[c->R]);
    return right ? gp_weno(c, f, c->wr, c->gr, beta) : gp_weno(c, f, c->wl, c->gl, beta);
}

/* The operation tally of a build with -DORACLE_COUNT_OPS (0 otherwise); reset
 * it to zero if asked. */
unsigned long long oracle_ops(int reset)
{
#ifdef ORACLE_COUNT_OPS
    unsigned long long v = g_ops;
    if (reset) g_ops = 0;
    return v;
#else
    (void)reset;
    return 0;
#endif
}
