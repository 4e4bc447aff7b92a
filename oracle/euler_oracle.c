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
 *     characteristic variables (Section 3.2-3.3; Section 6 for the use of
 *     characteristic variables): candidate predictions q^m = w_m^T f_m
 *     (Eq. candidate_interp), smoothness indicators beta_m = f_m^T K_m^{-1} f_m
 *     (Eq. gp-smooth, the definition form), WENO-JS weights
 *     omega_m = gamma_m/(eps+beta_m)^p normalised (Eq. weights), combination
 *     q = sum omega_m q^m (Eq. weight_sum);
 *   - the face flux F_{i+1/2} = RP(U^L, U^R) (Eq. riemann_prob) taken as the
 *     local Lax-Friedrichs (Rusanov) flux;
 *   - the high-order correction f^ = F + alpha D^2F + beta D^4F with
 *     alpha = -1/24, beta = 3/640 on neighbouring face fluxes (Eqs. numFlux_cor,
 *     FD-ders);
 *   - the semi-discrete divergence (Eq. disc_fd) and the three-stage SSP-RK
 *     update in Shu-Osher form (Section 2, step 5).
 *
 * Readings where the paper is silent: characteristic projection with the
 * eigenvectors of the Roe-averaged state of the two cells sharing the face,
 * in the textbook basis written out in roe_eigensystem() below; local
 * Lax-Friedrichs speed max(|u_n|+c) over U^L and U^R; ghost cells by periodic
 * wrap or zero-gradient copy, G = R+3 layers (R+1 for the face stencil, two
 * more for the correction).
 *
 * Layout: U is structure-of-arrays [nc][nz][ny][nx], nc = ndim+2 components
 * (rho, rho u_1..rho u_ndim, E), interior cells only, FP64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

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
}

/* Right (columns of Rm) and left (rows of Lm) eigenvectors of the flux Jacobian
 * in the normal direction at the Roe average of uL and uR (normal-first
 * ordering).  Textbook basis: acoustic u-c, entropy, one shear wave per
 * tangential velocity, acoustic u+c.  Returns 0 if the Roe state is not
 * physical. */
static int roe_eigensystem(const double *uL, const double *uR, int nc, double g,
                           double Rm[OR_MAXC][OR_MAXC], double Lm[OR_MAXC][OR_MAXC])
{
    int nv = nc - 2;            /* number of velocity components */
    double sL = sqrt(uL[0]), sR = sqrt(uR[0]);
    double vel[3], q2 = 0.0;
    double pL = pressure(uL, nc, g), pR = pressure(uR, nc, g);
    double HL = (uL[nc - 1] + pL) / uL[0], HR = (uR[nc - 1] + pR) / uR[0];
    for (int a = 0; a < nv; ++a) {
        vel[a] = (sL * uL[1 + a] / uL[0] + sR * uR[1 + a] / uR[0]) / (sL + sR);
        q2 += vel[a] * vel[a];
    }
    double H = (sL * HL + sR * HR) / (sL + sR);
    double c2 = (g - 1.0) * (H - 0.5 * q2);
    if (!(c2 > 0.0)) return 0;
    double c = sqrt(c2), un = vel[0];
    double b1 = (g - 1.0) / c2, b2 = 0.5 * q2 * b1;
    memset(Rm, 0, sizeof(double) * OR_MAXC * OR_MAXC);
    memset(Lm, 0, sizeof(double) * OR_MAXC * OR_MAXC);
    int E = nc - 1;
    /* wave 0: u - c */
    Rm[0][0] = 1.0; Rm[1][0] = un - c;
    for (int a = 1; a < nv; ++a) Rm[1 + a][0] = vel[a];
    Rm[E][0] = H - un * c;
    /* wave 1: entropy */
    Rm[0][1] = 1.0; Rm[1][1] = un;
    for (int a = 1; a < nv; ++a) Rm[1 + a][1] = vel[a];
    Rm[E][1] = 0.5 * q2;
    /* waves 2..nv: shear, one per tangential velocity */
    for (int t = 1; t < nv; ++t) { Rm[1 + t][1 + t] = 1.0; Rm[E][1 + t] = vel[t]; }
    /* wave nc-1: u + c */
    Rm[0][E] = 1.0; Rm[1][E] = un + c;
    for (int a = 1; a < nv; ++a) Rm[1 + a][E] = vel[a];
    Rm[E][E] = H + un * c;

    Lm[0][0] = 0.5 * (b2 + un / c);
    Lm[0][1] = 0.5 * (-b1 * un - 1.0 / c);
    for (int a = 1; a < nv; ++a) Lm[0][1 + a] = -0.5 * b1 * vel[a];
    Lm[0][E] = 0.5 * b1;
    Lm[1][0] = 1.0 - b2;
    for (int a = 0; a < nv; ++a) Lm[1][1 + a] = b1 * vel[a];
    Lm[1][E] = -b1;
    for (int t = 1; t < nv; ++t) { Lm[1 + t][0] = -vel[t]; Lm[1 + t][1 + t] = 1.0; }
    Lm[E][0] = 0.5 * (b2 - un / c);
    Lm[E][1] = 0.5 * (-b1 * un + 1.0 / c);
    for (int a = 1; a < nv; ++a) Lm[E][1 + a] = -0.5 * b1 * vel[a];
    Lm[E][E] = 0.5 * b1;
    return 1;
}

/* GP-WENO prediction at one face centre from 2R+1 values f[0..2R] centred on
 * the cell whose stencil is used; w: (R+1)x(R+1) sub-stencil weights, gam:
 * linear weights.  Sub-stencil m covers f[m..m+R] (Eq. sub-stencil). */
static double gp_weno(const oracle_cfg *c, const double *f, const double *w, const double *gam)
{
    int R = c->R, S = R + 1;
    double q[OR_MAXR + 1], wt[OR_MAXR + 1], wsum = 0.0, out = 0.0;
    for (int m = 0; m < S; ++m) {
        const double *fm = f + m;
        double qm = 0.0;
        for (int j = 0; j < S; ++j) qm += w[m * S + j] * fm[j];              /* Eq. candidate_interp */
        double beta = 0.0;                                                     /* Eq. gp-smooth */
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b) beta += fm[a] * c->Kinv[a * S + b] * fm[b];
        q[m] = qm;
        wt[m] = gam[m] / pow(c->eps + beta, (double)c->p);                     /* Eq. weights */
        wsum += wt[m];
    }
    for (int m = 0; m < S; ++m) out += (wt[m] / wsum) * q[m];                   /* Eq. weight_sum */
    return out;
}

/* Face flux F between cells s and s+1 along dimension d, at transverse
 * position (t1, t2) meaning the other two cell indices in natural order.
 * Writes nc values (natural component order).  Returns 0 on a non-physical
 * state. */
static int face_flux(const oracle_cfg *c, const double *U, int d, int s, const int cell[3], double *Fout,
                     double *uLout, double *uRout)
{
    int nc = c->ndim + 2, R = c->R, ns = 2 * R + 2;
    long N = ncells(c);
    /* component permutation to normal-first ordering */
    int perm[OR_MAXC];
    perm[0] = 0; perm[1] = 1 + d;
    int k = 2;
    for (int a = 0; a < c->ndim; ++a) if (a != d) perm[k++] = 1 + a;
    perm[nc - 1] = nc - 1;

    double st[OR_MAXS][OR_MAXC];           /* stencil, normal-first */
    for (int q = 0; q < ns; ++q) {
        int idx[3] = { cell[0], cell[1], cell[2] };
        idx[d] = map_index(c, d, s - R + q);
        long l = lin(c, idx[0], idx[1], idx[2]);
        for (int a = 0; a < nc; ++a) st[q][a] = U[(long)perm[a] * N + l];
    }
    double Rm[OR_MAXC][OR_MAXC], Lm[OR_MAXC][OR_MAXC];
    if (!roe_eigensystem(st[R], st[R + 1], nc, c->gamma, Rm, Lm)) return 0;

    /* characteristic projection of every stencil cell */
    double ch[OR_MAXC][OR_MAXS];
    for (int q = 0; q < ns; ++q)
        for (int f = 0; f < nc; ++f) {
            double acc = 0.0;
            for (int a = 0; a < nc; ++a) acc += Lm[f][a] * st[q][a];
            ch[f][q] = acc;
        }
    double wL[OR_MAXC], wR[OR_MAXC];
    for (int f = 0; f < nc; ++f) {
        wL[f] = gp_weno(c, &ch[f][0], c->wl, c->gl);   /* cells s-R..s+R, x* = +1/2 */
        wR[f] = gp_weno(c, &ch[f][1], c->wr, c->gr);   /* cells s+1-R..s+1+R, x* = -1/2 */
    }
    double uL[OR_MAXC], uR[OR_MAXC];
    for (int a = 0; a < nc; ++a) {
        double l = 0.0, r = 0.0;
        for (int f = 0; f < nc; ++f) { l += Rm[a][f] * wL[f]; r += Rm[a][f] * wR[f]; }
        uL[a] = l; uR[a] = r;
    }
    double pL = pressure(uL, nc, c->gamma), pR = pressure(uR, nc, c->gamma);
    if (!(uL[0] > 0.0) || !(uR[0] > 0.0) || !(pL > 0.0) || !(pR > 0.0)) return 0;
    double cL = sqrt(c->gamma * pL / uL[0]), cR = sqrt(c->gamma * pR / uR[0]);
    double aL = fabs(uL[1] / uL[0]) + cL, aR = fabs(uR[1] / uR[0]) + cR;
    double alpha = aL > aR ? aL : aR;
    double fL[OR_MAXC], fR[OR_MAXC];
    normal_flux(uL, nc, c->gamma, fL);
    normal_flux(uR, nc, c->gamma, fR);
    for (int a = 0; a < nc; ++a) {
        Fout[perm[a]] = 0.5 * (fL[a] + fR[a]) - 0.5 * alpha * (uR[a] - uL[a]);
        if (uLout) uLout[perm[a]] = uL[a];
        if (uRout) uRout[perm[a]] = uR[a];
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
    return F5[2] + A2 * D2 + A4 * D4;
}

double oracle_corrected_flux(const double *F5) { return corrected_flux(F5); }

/* dUdt = L(U), Eq. disc_fd with the corrected fluxes of Eq. numFlux_cor.
 * Returns 0 on success, 1 if any non-physical state was met. */
int oracle_rhs(const oracle_cfg *c, const double *U, double *dUdt)
{
    int nc = c->ndim + 2;
    long N = ncells(c);
    int bad = 0;
    memset(dUdt, 0, sizeof(double) * nc * N);
    for (int d = 0; d < c->ndim; ++d) {
        int n = c->n[d];
        int nf = n + 5;                     /* faces s = -3 .. n+1 */
        double *F = (double *)malloc(sizeof(double) * nf * nc);
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int b = 0; b < c->n[t2]; ++b)
            for (int a = 0; a < c->n[t1]; ++a) {
                int cell[3];
                cell[t1] = a; cell[t2] = b; cell[d] = 0;
                for (int s = -3; s <= n + 1; ++s)
                    if (!face_flux(c, U, d, s, cell, &F[(s + 3) * nc], NULL, NULL)) {
                        bad = 1;
                        for (int q = 0; q < nc; ++q) F[(s + 3) * nc + q] = NAN;
                    }
                for (int i = 0; i < n; ++i) {
                    cell[d] = i;
                    long l = lin(c, cell[0], cell[1], cell[2]);
                    for (int q = 0; q < nc; ++q) {
                        double fh[2];
                        for (int side = 0; side < 2; ++side) {
                            int s = i - 1 + side;   /* face s+1/2; F index of face t is t+3 */
                            double F5[5];
                            for (int e = 0; e < 5; ++e) F5[e] = F[(s + 1 + e) * nc + q];
                            fh[side] = corrected_flux(F5);
                        }
                        dUdt[(long)q * N + l] -= (fh[1] - fh[0]) / c->dx[d];
                    }
                }
            }
        free(F);
    }
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

/* Single face, exposed for unit tests: Riemann states and flux at the face
 * between stencil cells R and R+1 of a 1D stencil st[2R+2][nc] given in
 * natural order with the normal direction d.  Outputs uL, uR, F (nc each). */
int oracle_face(const oracle_cfg *c, int d, const double *st, double *uL, double *uR, double *F)
{
    /* Build a scratch grid of 2R+2 cells along d (others = 1) and reuse
     * face_flux on it so the unit test exercises the same code. */
    oracle_cfg g = *c;
    int ns = 2 * c->R + 2, nc = c->ndim + 2;
    for (int a = 0; a < 3; ++a) { g.n[a] = 1; g.bc_lo[a] = g.bc_hi[a] = 1; }
    g.n[d] = ns;
    double *U = (double *)malloc(sizeof(double) * ns * nc);
    for (int q = 0; q < ns; ++q)
        for (int a = 0; a < nc; ++a) U[(long)a * ns + q] = st[q * nc + a];
    int cell[3] = { 0, 0, 0 };
    int ok = face_flux(&g, U, d, c->R, cell, F, uL, uR);
    free(U);
    return ok;
}

/* Eigen-system at the Roe average of two states (normal-first ordering),
 * exposed for unit tests. */
int oracle_roe(int nc, double g, const double *uL, const double *uR, double *Rout, double *Lout)
{
    double Rm[OR_MAXC][OR_MAXC], Lm[OR_MAXC][OR_MAXC];
    int ok = roe_eigensystem(uL, uR, nc, g, Rm, Lm);
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) { Rout[a * nc + b] = Rm[a][b]; Lout[a * nc + b] = Lm[a][b]; }
    return ok;
}

/* GP-WENO prediction exposed for unit tests: f has 2R+1 values. */
double oracle_gp_weno(const oracle_cfg *c, const double *f, int right)
{
    return right ? gp_weno(c, f, c->wr, c->gr) : gp_weno(c, f, c->wl, c->gl);
}
