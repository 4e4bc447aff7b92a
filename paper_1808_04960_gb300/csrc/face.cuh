// Per-face GP-WENO evaluation on the device (sm_103a).
//
// One call computes, for one face between stencil cells R and R+1 of a
// (2R+2)-cell stencil along the face normal:
//   - the Roe average of the two cells sharing the face and the left/right
//     eigenvectors of the normal flux Jacobian there (characteristic
//     variables, Section 6 of the paper);
//   - the projection of every stencil cell on each characteristic field;
//   - per field, the GP-WENO left state (x* = x_i + dx/2 from the stencil of
//     cell i) and right state (x* = x_{i+1} - dx/2 from the stencil of cell
//     i+1): candidate predictions q^m = w_m . f_m (Eq. candidate_interp),
//     smoothness indicators beta = sum_h (P_h . f_m)^2 (Eq. beta-eigen, the
//     R+2 windows shared by both sides), nonlinear weights (Eq. weights) and
//     their combination (Eq. weight_sum);
//   - back-projection to conserved states U^L, U^R and the local
//     Lax-Friedrichs flux F = (F(U^L)+F(U^R))/2 - alpha (U^R-U^L)/2 with
//     alpha = max(|u_n|+c) over both states (Eq. riemann_prob).
// Stencil values arrive "normal-first": (rho, m_normal, m_tangential..., E).
//
// Nonlinear weights use the ratio form omega_m = gamma_m r_m^p / sum_s gamma_s r_s^p
// with r_m = b_min / b_m, b_m = eps + beta_m.  It equals Eq. weights
// exactly in real arithmetic and keeps (eps + beta)^p from underflowing in
// FP32 when beta -> 0 (eps = 1e-36 squared is below the FP32 range).
#pragma once
#include <cuda_runtime.h>

namespace gpweno {

template <typename T>
struct Num;

// FP32: single-instruction approximations (PTX rcp/rsqrt/sqrt .approx.ftz,
// about 1 ulp), enough for an FP32 path whose error budget is set by the
// stored FP32 state.
template <>
struct Num<float> {
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float rsqrt(float x)
    {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float sqrt(float x)
    {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float fabs(float x) { return fabsf(x); }
    static __device__ __forceinline__ float fmax(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float fmin(float a, float b) { return fminf(a, b); }
};

template <>
struct Num<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
    static __device__ __forceinline__ double fmax(double a, double b) { return ::fmax(a, b); }
    static __device__ __forceinline__ double fmin(double a, double b) { return ::fmin(a, b); }
};

// Weight tables of one plan in the arithmetic type.  Passed by value as a
// kernel parameter so every (warp-uniform) table read is a constant-bank
// operand.
template <typename T, int R>
struct FaceTables {
    T wl[R + 1][R + 1];   // sub-stencil weights, left state (x* = +1/2 from the stencil of cell s)
    T wr[R + 1][R + 1];   // sub-stencil weights, right state (x* = -1/2 from the stencil of cell s+1)
    T gl[R + 1];          // linear weights, left state
    T gr[R + 1];          // linear weights, right state
    T sl1[R + 1];         // sum_j wl[m][j] - 1
    T sr1[R + 1];         // sum_j wr[m][j] - 1
    T Ph[R + 1][(R + 2) / 2];  // P = v / sqrt(lambda) of K_m(sigma), half form, largest lambda first:
                               // even rows symmetric, odd rows skew (K_m is persymmetric)
    T Psum[R + 1];        // sum_j of each full row of P (zero for the skew rows)
    T eps;                // WENO epsilon
    T gamma;              // ratio of specific heats
    int p;                // WENO power, 1 or 2
};

// Nonlinear GP-WENO combination for one side: candidates q[m], beta windows b[m]
// (already eps + beta), linear weights g[m].  Ratio form of Eq. weights.
template <typename T, int R>
__device__ __forceinline__ T weno_combine(const T (&q)[R + 1], const T (&b)[R + 1], const T (&g)[R + 1], int p)
{
    T bmin = b[0];
#pragma unroll
    for (int m = 1; m <= R; ++m) bmin = Num<T>::fmin(bmin, b[m]);
    T num = T(0), den = T(0);
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        T r = bmin * Num<T>::rcp(b[m]);
        T w = g[m] * (p == 2 ? r * r : r);
        num = fma(w, q[m], num);
        den += w;
    }
    return num * Num<T>::rcp(den);
}

// Reference state of the "cell-relative" flux evaluation (normal-first order).
template <typename T, int NC>
struct RefState {
    T rho;            // density
    T m[NC - 2];      // momentum components
    T v[NC - 2];      // velocity components
    T p;              // pressure
    T hp;             // E + p
};

// G(w) = F(U_ref + w) - F(U_ref): normal flux perturbation for a state
// perturbation w, written so that every large quantity of the reference state
// multiplies a small one (no cancellation of O(1) fluxes):
//   dv_a = (w_m_a - v_a w_rho) / rho,        rho = rho_ref + w_rho
//   p'   = (gamma-1) (w_E - 1/2 sum_a (m_a dv_a + v_a w_m_a))
//   G    = (w_m_n,  m_n dv_n + v_n w_m_n + p',  m_t dv_n + v_n w_m_t,  v_n' (w_E + p') + dv_n (E+p)_ref)
// with m = m_ref + w_m and v_n' = v_n + dv_n.  Returns false if rho <= 0 or
// p <= 0 (or NaN) for the full state; `speed` = |u_n| + c of the full state.
template <typename T, int NC>
__device__ __forceinline__ bool pert_flux(const RefState<T, NC> &r, const T (&w)[NC], T gam, T (&G)[NC], T &speed)
{
    constexpr int NV = NC - 2, E = NC - 1;
    const T rho = r.rho + w[0];
    const T ir = Num<T>::rcp(rho);
    T dv[NV], m[NV];
    T k2 = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        dv[a] = fma(-r.v[a], w[0], w[1 + a]) * ir;
        m[a] = r.m[a] + w[1 + a];
        k2 = fma(m[a], dv[a], fma(r.v[a], w[1 + a], k2));
    }
    const T pp = (gam - T(1)) * fma(T(-0.5), k2, w[E]);
    const T vn = r.v[0] + dv[0];
    G[0] = w[1];
    G[1] = fma(m[0], dv[0], fma(r.v[0], w[1], pp));
#pragma unroll
    for (int a = 1; a < NV; ++a) G[1 + a] = fma(m[a], dv[0], r.v[0] * w[1 + a]);
    G[E] = fma(vn, w[E] + pp, dv[0] * r.hp);
    const T pr = r.p + pp;
    speed = Num<T>::fabs(vn) + Num<T>::sqrt(Num<T>::fmax(gam * pr * ir, T(1e-30)));
    return (rho > T(0)) && (pr > T(0));
}

// One face, cell-relative form.  st[0..2R+1] is the normal-first stencil; the
// face s+1/2 lies between st[R] (cell s) and st[R+1] (cell s+1).  Outputs
//   A = F_{s+1/2} - F(U_s)      (numerical face flux relative to cell s)
//   B = F(U_{s+1}) - F(U_s)     (physical flux difference of the two cells)
// so that the flux jump across cell s, F_{s+1/2} - F_{s-1/2} = A_s - A_{s-1} + B_{s-1},
// is formed from small quantities only.  In real arithmetic this is exactly
// the scheme (Roe-averaged characteristic projection, GP-WENO states by
// Eqs. candidate_interp, beta-eigen, weights, weight_sum, Lax-Friedrichs
// flux); the rewriting only changes where FP rounding falls:
//   * characteristic data are projected as differences d_j = L (U_j - U_s)
//     plus the centre value f_c = L U_s, so q^m = w_m . d_m + f_c sum_j w_mj and
//     P_h . f_m = P_h . d_m + f_c sum_j P_hj (the sums are precomputed);
//   * the left state is U_s + R (q_L - L U_s) and the right state
//     U_{s+1} + R (q_R - L U_{s+1}), using R L = I and sum_m omega_m = 1;
//   * fluxes are perturbations about U_s (pert_flux).
// Returns false on a non-physical Roe, left, right or neighbour state.
template <typename T, int NC, int R>
__device__ __forceinline__ bool face_rel(const T (&st)[2 * R + 2][NC], const FaceTables<T, R> &tb, T (&A)[NC],
                                         T (&B)[NC])
{
    constexpr int NS = 2 * R + 2;
    constexpr int E = NC - 1;
    constexpr int NV = NC - 2;
    constexpr int S = R + 1, HALF = S / 2;
    const T gm1 = tb.gamma - T(1);

    // --- Roe average of the two cells sharing the face -------------------
    const T rL = st[R][0], rR = st[R + 1][0];
    const T rsL = Num<T>::rsqrt(rL), rsR = Num<T>::rsqrt(rR);
    const T inv = Num<T>::rcp(rL * rsL + rR * rsR);  // 1/(sqrt(rhoL)+sqrt(rhoR))
    const T irL = rsL * rsL, irR = rsR * rsR;
    T vel[NV];
    T q2 = T(0), mL2 = T(0), mR2 = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        vel[a] = fma(st[R][1 + a], rsL, st[R + 1][1 + a] * rsR) * inv;
        q2 = fma(vel[a], vel[a], q2);
        mL2 = fma(st[R][1 + a], st[R][1 + a], mL2);
        mR2 = fma(st[R + 1][1 + a], st[R + 1][1 + a], mR2);
    }
    const T pL = gm1 * fma(T(-0.5) * mL2, irL, st[R][E]);
    const T pR = gm1 * fma(T(-0.5) * mR2, irR, st[R + 1][E]);
    const T H = fma(st[R][E] + pL, rsL, (st[R + 1][E] + pR) * rsR) * inv;
    const T c2 = gm1 * fma(T(-0.5), q2, H);
    bool ok = (rL > T(0)) && (rR > T(0)) && (c2 > T(0));
    const T ic = Num<T>::rsqrt(Num<T>::fmax(c2, T(1e-30)));
    const T c = c2 * ic;
    const T un = vel[0];
    const T b1 = gm1 * ic * ic;
    const T b2 = T(0.5) * q2 * b1;
    const T hb1 = T(0.5) * b1;

    // reference state: cell s
    RefState<T, NC> ref;
    ref.rho = rL;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        ref.m[a] = st[R][1 + a];
        ref.v[a] = st[R][1 + a] * irL;
    }
    ref.p = pL;
    ref.hp = st[R][E] + pL;

    // differences to cell s (D[R] is never used)
    T D[NS][NC];
#pragma unroll
    for (int j = 0; j < NS; ++j)
#pragma unroll
        for (int a = 0; a < NC; ++a) D[j][a] = (j == R) ? T(0) : st[j][a] - st[R][a];

    // row k of L applied to a state
    auto lrow = [&](int k, const T *u) -> T {
        if (k == 0 || k == E) {
            // acoustic rows: 1/2 (b2 +- un/c, -b1 un -+ 1/c, -b1 v_t, b1)
            const T sgn = (k == 0) ? T(1) : T(-1);
            T acc = fma(hb1, u[E], T(0.5) * fma(sgn * un, ic, b2) * u[0]);
            acc = fma(T(-0.5) * fma(b1, un, sgn * ic), u[1], acc);
#pragma unroll
            for (int a = 1; a < NV; ++a) acc = fma(-hb1 * vel[a], u[1 + a], acc);
            return acc;
        } else if (k == 1) {
            // entropy row: (1 - b2, b1 u_a..., -b1)
            T acc = fma(-b1, u[E], (T(1) - b2) * u[0]);
#pragma unroll
            for (int a = 0; a < NV; ++a) acc = fma(b1 * vel[a], u[1 + a], acc);
            return acc;
        }
        // shear row of tangential velocity k-1: (-v_t, ..., 1, ...)
        return fma(-vel[k - 1], u[0], u[k]);
    };

    T dqL[NC], dqR[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const T fc = lrow(k, st[R]);
        T d[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) d[j] = (j == R) ? T(0) : lrow(k, D[j]);

        // --- smoothness indicators on the R+2 windows d[w..w+R] --------
        T b[R + 2];
#pragma unroll
        for (int w = 0; w < R + 2; ++w) {
            T ps[HALF > 0 ? HALF : 1], ms[HALF > 0 ? HALF : 1];
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const int lo = w + j, hi = w + S - 1 - j;
                ps[j] = lo == R ? d[hi] : (hi == R ? d[lo] : d[lo] + d[hi]);
                ms[j] = lo == R ? -d[hi] : (hi == R ? d[lo] : d[lo] - d[hi]);
            }
            T beta = T(0);
#pragma unroll
            for (int h = 0; h < S; ++h) {
                T dot;
                if (h % 2 == 0) {
                    dot = tb.Psum[h] * fc;
                    if (S % 2 == 1 && w + HALF != R) dot = fma(tb.Ph[h][HALF], d[w + HALF], dot);
#pragma unroll
                    for (int j = 0; j < HALF; ++j) dot = fma(tb.Ph[h][j], ps[j], dot);
                } else {
                    dot = tb.Ph[h][0] * ms[0];
#pragma unroll
                    for (int j = 1; j < HALF; ++j) dot = fma(tb.Ph[h][j], ms[j], dot);
                }
                beta = fma(dot, dot, beta);
            }
            b[w] = tb.eps + beta;
        }
        // --- candidates relative to the centre cells, both sides ---------
        T cl[R + 1], cr[R + 1], bl[R + 1], br[R + 1];
#pragma unroll
        for (int m = 0; m <= R; ++m) {
            T sl = tb.sl1[m] * fc, sr = tb.sr1[m] * fc;
#pragma unroll
            for (int j = 0; j <= R; ++j) {
                if (m + j != R) sl = fma(tb.wl[m][j], d[m + j], sl);
                if (1 + m + j != R) sr = fma(tb.wr[m][j], d[1 + m + j], sr);
            }
            cl[m] = sl;
            cr[m] = sr;
            bl[m] = b[m];
            br[m] = b[m + 1];
        }
        dqL[k] = weno_combine<T, R>(cl, bl, tb.gl, tb.p);              // q_L - L U_s
        dqR[k] = weno_combine<T, R>(cr, br, tb.gr, tb.p) - d[R + 1];   // q_R - L U_{s+1}
    }

    // --- back-projection: states relative to cell s -----------------------
    T uL[NC], uR[NC];
    {
        const T hL = dqL[0] + dqL[1] + dqL[E], hR = dqR[0] + dqR[1] + dqR[E];
        const T aL = c * (dqL[E] - dqL[0]), aR = c * (dqR[E] - dqR[0]);
        uL[0] = hL;
        uR[0] = D[R + 1][0] + hR;
        uL[1] = fma(un, hL, aL);
        uR[1] = D[R + 1][1] + fma(un, hR, aR);
        T eL = fma(H, dqL[0] + dqL[E], fma(T(0.5) * q2, dqL[1], un * aL));
        T eR = fma(H, dqR[0] + dqR[E], fma(T(0.5) * q2, dqR[1], un * aR));
#pragma unroll
        for (int a = 1; a < NV; ++a) {
            uL[1 + a] = fma(vel[a], hL, dqL[1 + a]);
            uR[1 + a] = D[R + 1][1 + a] + fma(vel[a], hR, dqR[1 + a]);
            eL = fma(vel[a], dqL[1 + a], eL);
            eR = fma(vel[a], dqR[1 + a], eR);
        }
        uL[E] = eL;
        uR[E] = D[R + 1][E] + eR;
    }

    // --- Lax-Friedrichs flux relative to F(U_s), and F(U_{s+1}) - F(U_s) ----
    T GL[NC], GR[NC], sL, sR, sB;
    ok = pert_flux<T, NC>(ref, uL, tb.gamma, GL, sL) && ok;
    ok = pert_flux<T, NC>(ref, uR, tb.gamma, GR, sR) && ok;
    T dn[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) dn[a] = D[R + 1][a];
    ok = pert_flux<T, NC>(ref, dn, tb.gamma, B, sB) && ok;
    const T alpha = Num<T>::fmax(sL, sR);
#pragma unroll
    for (int a = 0; a < NC; ++a) A[a] = T(0.5) * ((GL[a] + GR[a]) - alpha * (uR[a] - uL[a]));
    return ok;
}

// Weights of the corrected-flux difference: with the face-flux correction
// f^_{s+1/2} = F + alpha D2F + beta D4F (Eqs. numFlux_cor, FD-ders; alpha = -1/24,
// beta = 3/640), f^_{i+1/2} - f^_{i-1/2} = sum_{k=-2..2} c_k dF_{i+k} where
// dF_s = F_{s+1/2} - F_{s-1/2} and c = (beta, alpha-4beta, 1-2alpha+6beta, alpha-4beta, beta).
template <typename T>
__device__ __forceinline__ T corrected_divergence(T d0, T d1, T d2, T d3, T d4)
{
    constexpr double al = -1.0 / 24.0, be = 3.0 / 640.0;
    const T c0 = T(be), c1 = T(al - 4.0 * be), c2 = T(1.0 - 2.0 * al + 6.0 * be);
    return fma(c0, d0 + d4, fma(c1, d1 + d3, c2 * d2));
}

// Index of cell i along a dimension of n cells after the boundary map:
// periodic wrap or zero-gradient clamp (outflow).  Periodic wrap is a full
// modulo, so grids narrower than the ghost width are handled.
__device__ __forceinline__ int bc_map(int i, int n, int periodic)
{
    if (i >= 0 && i < n) return i;
    if (periodic) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    return i < 0 ? 0 : n - 1;
}

}  // namespace gpweno
