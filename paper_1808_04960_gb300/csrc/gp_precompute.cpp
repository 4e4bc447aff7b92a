// GP-WENO weight tables in double-double arithmetic.
//
// Section 4, step 1 of the paper: covariance matrices K (full stencil) and
// K_m (sub-stencils) of the squared-exponential kernel (Eqs. se, kmat), the
// prediction vectors k* (Eq. kstar), the GP weights w = K^{-1} k* and
// w_m = K_m^{-1} k*_m (Eqs. q-intrp, candidate_interp), the linear weights
// gamma as the least-squares solution of M gamma = w (Eqs. gamm-system,
// M-mat), and the eigen-system of K_m built with sigma, giving
// P_h = v_h / sqrt(lambda_h) for beta_m = sum_h (P_h . f_m)^2 (Eq. beta-eigen).
//
// K is severely ill-conditioned at large l/dx (about 8e13 at R=3, l/dx=12 and
// 3e17 at l/dx=24), so FP64 alone cannot produce FP64-accurate weights.  All
// arithmetic here is double-double (Dekker 1971; Knuth's TwoSum; TwoProd via
// fma), about 32 significant digits, portable across x86-64 and aarch64.
//
// Every kernel entry is exp(-(a-b)^2 / (2 l^2)) with a-b a multiple of 1/2 (in
// units of dx), i.e. q^n with q = exp(-1/(8 l^2)) and the integer n =
// 4 (a-b)^2.  So a single exponential is evaluated (Taylor series after
// halving the argument, squared back) and every entry is an exact-integer
// power of q, which keeps all entries accurate to a few units of 2^-104.
//
// Reconstruction tables (FD-Flux form, Section 2: the point fluxes are cell
// averages of the function whose face values are wanted, Eqs. prim_F and
// design) condition the GP on cell averages.  Their covariances are power
// series in a = 1/(2 l^2) with exact-integer coefficients (see cavg_cov and
// point_cell_cov), summed in double-double.
#include "gp_precompute.h"

#include <cmath>
#include <cstdio>
#include <cstring>

namespace gpweno {
namespace {

struct dd {
    double hi, lo;
};

inline dd make(double a) { return {a, 0.0}; }

inline dd two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

inline dd quick_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}

inline dd two_prod(double a, double b)
{
    double p = a * b;
    double e = std::fma(a, b, -p);
    return {p, e};
}

inline dd add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }

inline dd mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

inline dd mul_d(dd a, double b)
{
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}

inline dd div(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = sub(a, mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = sub(r, mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return add(q, make(q3));
}

// sqrt by one Newton step in double-double from the FP64 root.
inline dd sqrt_dd(dd a)
{
    if (a.hi <= 0.0) return make(0.0);
    double x = std::sqrt(a.hi);
    dd xx = two_prod(x, x);
    dd r = sub(a, xx);
    return add(make(x), make(r.hi / (2.0 * x)));
}

inline double to_d(dd a) { return a.hi + a.lo; }

// exp(y) for y <= 0 of moderate size: halve the argument s times so that
// |y / 2^s| <= 1/16, sum the Taylor series to 2^-110, then square s times.
dd exp_dd(dd y)
{
    int s = 0;
    dd z = y;
    while (std::fabs(z.hi) > 1.0 / 16.0) {
        z = mul_d(z, 0.5);
        ++s;
    }
    dd term = make(1.0), sum = make(1.0);
    for (int k = 1; k < 40; ++k) {
        term = div(mul(term, z), make((double)k));
        sum = add(sum, term);
        if (std::fabs(term.hi) < 1e-40) break;
    }
    for (int k = 0; k < s; ++k) sum = mul(sum, sum);
    return sum;
}

dd pow_int(dd q, int n)
{
    dd r = make(1.0), b = q;
    while (n > 0) {
        if (n & 1) r = mul(r, b);
        b = mul(b, b);
        n >>= 1;
    }
    return r;
}

// Entry of the SE kernel between points a/2 and b/2 (half-integer grid, units
// of dx) given q = exp(-1/(8 l^2)):  exp(-((a-b)/2)^2 / (2 l^2)) = q^((a-b)^2).
dd se_entry(dd q, int a2, int b2)
{
    int d = a2 - b2;
    return pow_int(q, d * d);
}

// b^e for small integers (either sign), exact in double-double while below 2^106.
dd ipow(int b, int e)
{
    dd r = make(1.0);
    for (int k = 0; k < e; ++k) r = mul_d(r, (double)b);
    return r;
}

// Covariance of the averages over two unit cells whose centres are delta apart
// (units of dx) under exp(-a u^2):
//   C(delta) = int_{-1}^{1} (1 - |t|) exp(-a (delta + t)^2) dt
//            = sum_n (-a)^n / n! * [(delta+1)^(2n+2) - 2 delta^(2n+2) + (delta-1)^(2n+2)] / ((2n+1)(2n+2)),
// the bracket being the second difference of the second antiderivative of u^(2n).
dd cavg_cov(dd a, int delta)
{
    if (delta < 0) delta = -delta;
    const double xmax = delta + 1.0;
    dd coef = make(1.0), sum = make(0.0);
    for (int n = 0; n < 400; ++n) {
        if (n > 0) coef = div(mul(coef, neg(a)), make((double)n));
        const int e = 2 * n + 2;
        dd m = add(sub(ipow(delta + 1, e), mul_d(ipow(delta, e), 2.0)), ipow(delta - 1, e));
        dd term = div(mul(coef, m), make((double)(2 * n + 1) * (double)(2 * n + 2)));
        sum = add(sum, term);
        if (n > a.hi * xmax * xmax + 4 && std::fabs(term.hi) < 1e-36 * std::fabs(sum.hi)) break;
    }
    return sum;
}

// Covariance of the point value at offset u = u2/2 (u2 odd, units of dx) from a cell
// centre with the average over that unit cell:
//   T(u) = int_{-1/2}^{1/2} exp(-a (u + t)^2) dt
//        = sum_n (-a)^n / n! * [(u+1/2)^(2n+1) - (u-1/2)^(2n+1)] / (2n+1).
dd point_cell_cov(dd a, int u2)
{
    const int hi = (u2 + 1) / 2, lo = (u2 - 1) / 2;   // u + 1/2 and u - 1/2, integers
    const double xmax = std::fmax(std::fabs((double)hi), std::fabs((double)lo));
    dd coef = make(1.0), sum = make(0.0);
    for (int n = 0; n < 400; ++n) {
        if (n > 0) coef = div(mul(coef, neg(a)), make((double)n));
        const int e = 2 * n + 1;
        dd term = div(mul(coef, sub(ipow(hi, e), ipow(lo, e))), make((double)(2 * n + 1)));
        sum = add(sum, term);
        if (n > a.hi * xmax * xmax + 4 && std::fabs(term.hi) < 1e-36 * std::fabs(sum.hi)) break;
    }
    return sum;
}

// Polynomial reconstruction at xs2/2 from averages over unit cells centred at
// pts2[j]/2: the primitive function at the n+1 cell edges is interpolated and
// differentiated, w_j = sum_{m>j} L'_m(x*) with L_m the Lagrange basis on the edges.
void poly_recon_weights(const int *pts2, int n, int xs2, dd *w)
{
    int e2[kMaxBig + 1];                 // edges in half-units
    e2[0] = pts2[0] - 1;
    for (int j = 0; j < n; ++j) e2[j + 1] = pts2[j] + 1;
    const int ne = n + 1;
    dd dL[kMaxBig + 1];
    for (int m = 0; m < ne; ++m) {
        dd den = make(1.0);
        for (int l = 0; l < ne; ++l)
            if (l != m) den = mul_d(den, 0.5 * (e2[m] - e2[l]));
        dd num = make(0.0);
        for (int l = 0; l < ne; ++l) {
            if (l == m) continue;
            dd prod = make(1.0);
            for (int q = 0; q < ne; ++q)
                if (q != m && q != l) prod = mul_d(prod, 0.5 * (xs2 - e2[q]));
            num = add(num, prod);
        }
        dL[m] = div(num, den);
    }
    for (int j = 0; j < n; ++j) {
        dd s = make(0.0);
        for (int m = j + 1; m < ne; ++m) s = add(s, dL[m]);
        w[j] = s;
    }
}

// Cholesky factorisation A = C C^T (lower C) and solves, n <= kMaxBig.
struct Chol {
    int n;
    dd C[kMaxBig][kMaxBig];
    bool ok;
    double cond_est;
};

Chol cholesky(const dd A[kMaxBig][kMaxBig], int n)
{
    Chol ch;
    ch.n = n;
    ch.ok = true;
    std::memset(ch.C, 0, sizeof(ch.C));
    double dmax = 0.0, dmin = 1e300;
    for (int j = 0; j < n; ++j) {
        dd s = A[j][j];
        for (int k = 0; k < j; ++k) s = sub(s, mul(ch.C[j][k], ch.C[j][k]));
        if (!(s.hi > 0.0)) {
            ch.ok = false;
            ch.cond_est = INFINITY;
            return ch;
        }
        ch.C[j][j] = sqrt_dd(s);
        double dj = std::fabs(ch.C[j][j].hi);
        if (dj > dmax) dmax = dj;
        if (dj < dmin) dmin = dj;
        for (int i = j + 1; i < n; ++i) {
            dd t = A[i][j];
            for (int k = 0; k < j; ++k) t = sub(t, mul(ch.C[i][k], ch.C[j][k]));
            ch.C[i][j] = div(t, ch.C[j][j]);
        }
    }
    ch.cond_est = (dmax / dmin) * (dmax / dmin);
    return ch;
}

void chol_solve(const Chol &ch, const dd *b, dd *x)
{
    int n = ch.n;
    dd y[kMaxBig];
    for (int i = 0; i < n; ++i) {
        dd s = b[i];
        for (int k = 0; k < i; ++k) s = sub(s, mul(ch.C[i][k], y[k]));
        y[i] = div(s, ch.C[i][i]);
    }
    for (int i = n - 1; i >= 0; --i) {
        dd s = y[i];
        for (int k = i + 1; k < n; ++k) s = sub(s, mul(ch.C[k][i], x[k]));
        x[i] = div(s, ch.C[i][i]);
    }
}

// Lagrange interpolation weights at xs2 for the points pts2 (half-units):
// l_j = prod_{k != j} (xs2 - p_k) / (p_j - p_k), ratios of small integers.
void lagrange_weights(const int *pts2, int n, int xs2, dd *w)
{
    for (int j = 0; j < n; ++j) {
        dd v = make(1.0);
        for (int k = 0; k < n; ++k)
            if (k != j) v = div(mul_d(v, (double)(xs2 - pts2[k])), make((double)(pts2[j] - pts2[k])));
        w[j] = v;
    }
}

// Prediction weights for the points 2*p2[k] (half-units) and the prediction
// point xs2 (half-units).  Point data: GP weights w = K^{-1} k*, or with
// `poly` Lagrange weights.  Cell-average data (`recon`, a = 1/(2 l^2)): GP
// weights w = C^{-1} T, or with `poly` polynomial reconstruction weights.
struct WeightKind {
    int poly, recon;
    dd a;
};

bool gp_weights(dd q, const int *pts2, int n, int xs2, dd *w, double *cond, const WeightKind &kind)
{
    if (kind.poly) {
        if (kind.recon) poly_recon_weights(pts2, n, xs2, w);
        else lagrange_weights(pts2, n, xs2, w);
        if (cond) *cond = 1.0;
        return true;
    }
    dd K[kMaxBig][kMaxBig];
    dd ks[kMaxBig];
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b)
            K[a][b] = kind.recon ? cavg_cov(kind.a, (pts2[a] - pts2[b]) / 2) : se_entry(q, pts2[a], pts2[b]);
        ks[a] = kind.recon ? point_cell_cov(kind.a, xs2 - pts2[a]) : se_entry(q, xs2, pts2[a]);
    }
    Chol ch = cholesky(K, n);
    if (cond) *cond = ch.cond_est;
    if (!ch.ok) return false;
    chol_solve(ch, ks, w);
    return true;
}

// Cyclic Jacobi eigen-decomposition of a small symmetric matrix in
// double-double; textbook rotations (Golub & Van Loan, Alg. 8.4.2).
void jacobi(dd A[kMaxBig][kMaxBig], int n, dd V[kMaxBig][kMaxBig])
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i][j] = make(i == j ? 1.0 : 0.0);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i != j) off += A[i][j].hi * A[i][j].hi;
                else diag += A[i][j].hi * A[i][j].hi;
            }
        // double-double rounding leaves off-diagonal entries near 1e-32 relative
        if (off <= 1e-60 * diag) break;
        for (int p = 0; p < n - 1; ++p)
            for (int r = p + 1; r < n; ++r) {
                if (std::fabs(A[p][r].hi) <= 1e-34 * (std::fabs(A[p][p].hi) + std::fabs(A[r][r].hi))) continue;
                dd theta = div(sub(A[r][r], A[p][p]), mul_d(A[p][r], 2.0));
                dd root = sqrt_dd(add(mul(theta, theta), make(1.0)));
                dd t = theta.hi >= 0.0 ? div(make(1.0), add(theta, root)) : div(make(-1.0), sub(root, theta));
                dd c = div(make(1.0), sqrt_dd(add(mul(t, t), make(1.0))));
                dd s = mul(t, c);
                for (int k = 0; k < n; ++k) {
                    dd akp = A[k][p], akr = A[k][r];
                    A[k][p] = sub(mul(c, akp), mul(s, akr));
                    A[k][r] = add(mul(s, akp), mul(c, akr));
                }
                for (int k = 0; k < n; ++k) {
                    dd apk = A[p][k], ark = A[r][k];
                    A[p][k] = sub(mul(c, apk), mul(s, ark));
                    A[r][k] = add(mul(s, apk), mul(c, ark));
                }
                for (int k = 0; k < n; ++k) {
                    dd vkp = V[k][p], vkr = V[k][r];
                    V[k][p] = sub(mul(c, vkp), mul(s, vkr));
                    V[k][r] = add(mul(s, vkp), mul(c, vkr));
                }
            }
    }
}

// Linear weights for one prediction point: sub-stencil weights, full-stencil
// weights, then least squares of M gamma = w through the normal equations.
bool side_tables(dd q, int R, int xs2, double *w_sub, double *w_big, double *gam, double *resid, double *cond,
                 double *sum1, char *err, std::size_t errlen, const WeightKind &kind)
{
    const int S = R + 1, B = 2 * R + 1;
    int big2[kMaxBig];
    for (int j = 0; j < B; ++j) big2[j] = 2 * (j - R);
    dd wb[kMaxBig];
    if (!gp_weights(q, big2, B, xs2, wb, cond, kind)) {
        std::snprintf(err, errlen, "covariance K of the %d-point stencil is not positive definite in double-double", B);
        return false;
    }
    dd ws[kMaxS][kMaxS];
    for (int m = 0; m < S; ++m) {
        int p2[kMaxS];
        for (int j = 0; j < S; ++j) p2[j] = 2 * (-R + m + j);
        if (!gp_weights(q, p2, S, xs2, ws[m], nullptr, kind)) {
            std::snprintf(err, errlen, "sub-stencil covariance K_m is not positive definite in double-double");
            return false;
        }
    }
    // M: (2R+1) x (R+1), column n holds w_n in rows n..n+R (Eq. M-mat)
    dd M[kMaxBig][kMaxS];
    for (int r = 0; r < B; ++r)
        for (int c = 0; c < S; ++c) M[r][c] = make(0.0);
    for (int c = 0; c < S; ++c)
        for (int j = 0; j < S; ++j) M[c + j][c] = ws[c][j];
    dd N[kMaxBig][kMaxBig], rhs[kMaxBig], g[kMaxBig];
    for (int a = 0; a < S; ++a) {
        for (int b = 0; b < S; ++b) {
            dd s = make(0.0);
            for (int r = 0; r < B; ++r) s = add(s, mul(M[r][a], M[r][b]));
            N[a][b] = s;
        }
        dd s = make(0.0);
        for (int r = 0; r < B; ++r) s = add(s, mul(M[r][a], wb[r]));
        rhs[a] = s;
    }
    Chol ch = cholesky(N, S);
    if (!ch.ok) {
        std::snprintf(err, errlen, "normal equations of the linear-weight system are singular");
        return false;
    }
    chol_solve(ch, rhs, g);
    double r2 = 0.0;
    for (int r = 0; r < B; ++r) {
        dd s = neg(wb[r]);
        for (int c = 0; c < S; ++c) s = add(s, mul(M[r][c], g[c]));
        r2 += to_d(s) * to_d(s);
    }
    *resid = std::sqrt(r2);
    for (int m = 0; m < S; ++m)
        for (int j = 0; j < S; ++j) w_sub[m * S + j] = to_d(ws[m][j]);
    for (int j = 0; j < B; ++j) w_big[j] = to_d(wb[j]);
    for (int m = 0; m < S; ++m) gam[m] = to_d(g[m]);
    for (int m = 0; m < S; ++m) {
        dd acc = make(-1.0);
        for (int j = 0; j < S; ++j) acc = add(acc, ws[m][j]);
        sum1[m] = to_d(acc);
    }
    return true;
}

// Smoothness factors of the N-point covariance K_N(sigma) (points 0..N-1):
// P[h*N + j] = v_h[j] / sqrt(lambda_h) with lambda ascending, the half form
// Ph[k*N + j] (j < (N+1)/2, largest lambda first, symmetric and skew rows
// alternating -- checked), the row sums Psum (zero for skew rows) and
// log det K_N.
bool eigen_factors(dd qs, int N, double *P, double *lambda, double *Ph, double *Psum, double *logdet, char *err,
                   std::size_t errlen, double *one_kinv_one = nullptr)
{
    dd Ks[kMaxBig][kMaxBig], V[kMaxBig][kMaxBig];
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) Ks[a][b] = se_entry(qs, 2 * a, 2 * b);
    jacobi(Ks, N, V);
    int order[kMaxBig];
    for (int h = 0; h < N; ++h) order[h] = h;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            if (Ks[order[b]][order[b]].hi < Ks[order[a]][order[a]].hi) {
                int t = order[a];
                order[a] = order[b];
                order[b] = t;
            }
    double ld = 0.0;
    dd ones = make(0.0);   // 1^T K^-1 1 = sum_h (v_h . 1)^2 / lambda_h
    for (int h = 0; h < N; ++h) {
        int e = order[h];
        dd lam = Ks[e][e];
        if (!(lam.hi > 0.0)) {
            std::snprintf(err, errlen, "K_%d(sigma) has a non-positive eigenvalue", N);
            return false;
        }
        lambda[h] = to_d(lam);
        ld += std::log(lambda[h]);
        dd rs = div(make(1.0), sqrt_dd(lam));
        dd vs = make(0.0);
        for (int j = 0; j < N; ++j) {
            P[h * N + j] = to_d(mul(V[j][e], rs));
            vs = add(vs, V[j][e]);
        }
        ones = add(ones, div(mul(vs, vs), lam));
    }
    if (one_kinv_one) *one_kinv_one = to_d(ones);
    if (logdet) *logdet = ld;
    // half form, descending lambda, with the symmetric/skew alternation checked
    for (int k = 0; k < N; ++k) {
        const double *row = P + (N - 1 - k) * N;
        double scale = 0.0;
        for (int j = 0; j < N; ++j) scale = std::fmax(scale, std::fabs(row[j]));
        const double sgn = (k % 2 == 0) ? 1.0 : -1.0;
        for (int j = 0; j < N; ++j)
            if (std::fabs(row[j] - sgn * row[N - 1 - j]) > 1e-12 * scale) {
                std::snprintf(err, errlen, "eigenvector %d of K_%d(sigma) is not %s", k, N,
                              k % 2 == 0 ? "symmetric" : "skew-symmetric");
                return false;
            }
        for (int j = 0; j < (N + 1) / 2; ++j) Ph[k * N + j] = row[j];
        dd sum = make(0.0);
        for (int j = 0; j < N; ++j) sum = add(sum, make(row[j]));
        Psum[k] = (k % 2 == 0) ? to_d(sum) : 0.0;
    }
    return true;
}

}  // namespace

int gp_precompute(int R, double ell, double sigma, GpTables *out, char *err, std::size_t errlen, int poly, int recon)
{
    if (R < 1 || R > kMaxR) {
        std::snprintf(err, errlen, "R=%d out of range [1,%d]", R, kMaxR);
        return 1;
    }
    if (!(ell >= 1.0) || !(ell <= 1.0e3)) {
        std::snprintf(err, errlen, "l/dx=%g out of range [1,1000]", ell);
        return 1;
    }
    if (!(sigma > 1.0) || !(sigma <= 1.0e3)) {
        std::snprintf(err, errlen, "sigma/dx=%g out of range (1,1000] (sigma <= dx is unstable, Section 3.4)", sigma);
        return 1;
    }
    std::memset(out, 0, sizeof(*out));
    out->R = R;
    const int S = R + 1;
    // q = exp(-1/(8 l^2)) in double-double; 1/(8 l^2) formed exactly enough by a dd division
    dd ql = exp_dd(neg(div(make(1.0), mul_d(mul(make(ell), make(ell)), 8.0))));
    dd qs = exp_dd(neg(div(make(1.0), mul_d(mul(make(sigma), make(sigma)), 8.0))));
    WeightKind kind;
    kind.poly = poly;
    kind.recon = recon;
    kind.a = div(make(0.5), mul(make(ell), make(ell)));
    double cond = 0.0, resid_r = 0.0;
    if (!side_tables(ql, R, +1, out->wl, out->wbig_l, out->gl, &out->ls_residual, &cond, out->sl1, err, errlen, kind))
        return 2;
    if (!side_tables(ql, R, -1, out->wr, out->wbig_r, out->gr, &resid_r, nullptr, out->sr1, err, errlen, kind))
        return 2;
    out->cond_estimate = cond;
    for (int m = 0; m < S; ++m) {
        for (int j = 0; j < S; ++j) {
            out->gwl[m * S + j] = out->gl[m] * out->wl[m * S + j];
            out->gwr[m * S + j] = out->gr[m] * out->wr[m * S + j];
        }
        out->gsl1[m] = out->gl[m] * out->sl1[m];
        out->gsr1[m] = out->gr[m] * out->sr1[m];
    }
    // double-double carries ~2^-104 relative; demand cond * 2^-104 < 1e-6
    if (cond * 4.93e-32 > 1e-6) {
        std::snprintf(err, errlen, "covariance of R=%d at l/dx=%g has condition ~%.3g, beyond double-double", R, ell,
                      cond);
        return 2;
    }
    // smoothness-indicator covariance K_m(sigma) on the points 0..R
    if (!eigen_factors(qs, S, out->P, out->lambda, out->Ph, out->Psum, nullptr, err, errlen)) return 2;
    return 0;
}

int ao_precompute(int R, double ell, double sigma, AoTables *out, char *err, std::size_t errlen)
{
    if (R != 2 && R != 3) {
        std::snprintf(err, errlen, "GP-AO needs R = 2 (AO(2,3)) or R = 3 (AO(3,2,3)), got %d", R);
        return 1;
    }
    std::memset(out, 0, sizeof(*out));
    out->R = R;
    dd ql = exp_dd(neg(div(make(1.0), mul_d(mul(make(ell), make(ell)), 8.0))));
    dd qs = exp_dd(neg(div(make(1.0), mul_d(mul(make(sigma), make(sigma)), 8.0))));
    WeightKind kind;
    kind.poly = 0;
    kind.recon = 0;
    kind.a = make(0.0);
    // GP weights of one stencil (cells lo..hi relative to the centre) at x* = +-1/2, and sum - 1
    auto weights = [&](int lo, int hi, double *wl, double *wr, double *sl, double *sr) {
        int p2[kMaxBig];
        const int n = hi - lo + 1;
        for (int j = 0; j < n; ++j) p2[j] = 2 * (lo + j);
        dd w[kMaxBig];
        for (int side = 0; side < 2; ++side) {
            if (!gp_weights(ql, p2, n, side == 0 ? 1 : -1, w, nullptr, kind)) return false;
            dd acc = make(-1.0);
            for (int j = 0; j < n; ++j) {
                (side == 0 ? wl : wr)[j] = to_d(w[j]);
                acc = add(acc, w[j]);
            }
            *(side == 0 ? sl : sr) = to_d(acc);
        }
        return true;
    };
    bool ok = weights(-R, R, out->w_hi_l, out->w_hi_r, &out->s_hi_l, &out->s_hi_r);
    if (R == 3) ok = ok && weights(-(R - 1), R - 1, out->w_lo_l, out->w_lo_r, &out->s_lo_l, &out->s_lo_r);
    for (int m = 0; m < 3; ++m)   // Eq. cweno_stencil: cells i-2..i, i-1..i+1, i..i+2
        ok = ok && weights(m - 2, m, out->w3_l + 3 * m, out->w3_r + 3 * m, out->s3_l + m, out->s3_r + m);
    if (!ok) {
        std::snprintf(err, errlen, "a GP-AO stencil covariance is not positive definite in double-double");
        return 2;
    }
    // Stencils of different size are compared through the data-fit term per unit of that of
    // constant data: beta_N = f^T K_N^-1 f / (1^T K_N^-1 1), so that smooth data give every
    // stencil nearly the same indicator; dividing beta by 1^T K_N^-1 1 (double-double) scales the
    // factors P by its inverse square root.
    double lam[kMaxBig], one_hi = 1.0, one_lo = 1.0, one_3 = 1.0;
    if (!eigen_factors(qs, 2 * R + 1, out->P_hi, lam, out->Ph_hi, out->Psum_hi, &out->logdet_hi, err, errlen,
                       &one_hi))
        return 2;
    if (R == 3 && !eigen_factors(qs, 2 * R - 1, out->P_lo, lam, out->Ph_lo, out->Psum_lo, &out->logdet_lo, err,
                                 errlen, &one_lo))
        return 2;
    if (!eigen_factors(qs, 3, out->P_3, lam, out->Ph_3, out->Psum_3, &out->logdet_3, err, errlen, &one_3)) return 2;
    auto normalise = [](int N, double one, double *P, double *Ph, double *Psum) {
        const double s = 1.0 / std::sqrt(one);
        for (int k = 0; k < N * N; ++k) {
            P[k] *= s;
            Ph[k] *= s;
        }
        for (int h = 0; h < N; ++h) Psum[h] *= s;
    };
    normalise(2 * R + 1, one_hi, out->P_hi, out->Ph_hi, out->Psum_hi);
    if (R == 3) normalise(2 * R - 1, one_lo, out->P_lo, out->Ph_lo, out->Psum_lo);
    normalise(3, one_3, out->P_3, out->Ph_3, out->Psum_3);
    return 0;
}

}  // namespace gpweno
