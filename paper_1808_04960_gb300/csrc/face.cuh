// Per-face GP-WENO evaluation on the device (sm_103a).
//
// One call computes, for one face between stencil cells R and R+1 of a
// (2R+2)-cell stencil along the face normal:
//   - the Roe average of the two cells sharing the face and the left/right
//     eigenvectors of the primitive-variable system there (characteristic
//     variables of V = (rho, u, p), Section 6 of the paper);
//   - the projection of every stencil cell's primitive variables on each
//     characteristic field;
//   - per field, the GP-WENO left state (x* = x_i + dx/2 from the stencil of
//     cell i) and right state (x* = x_{i+1} - dx/2 from the stencil of cell
//     i+1): candidate predictions q^m = w_m . f_m (Eq. candidate_interp),
//     smoothness indicators beta = sum_h (P_h . f_m)^2 (Eq. beta-eigen, the
//     R+2 windows shared by both sides), nonlinear weights (Eq. weights) and
//     their combination (Eq. weight_sum);
//   - back-projection to the Riemann states U^L, U^R and the face flux of
//     Eq. riemann_prob: local Lax-Friedrichs, F = (F(U^L)+F(U^R))/2 -
//     alpha (U^R-U^L)/2 with alpha = max(|u_n|+c) over both states, or HLLC
//     (the paper's default solver, Section 7) with Einfeldt wave speeds.
// Stencil values arrive conserved and "normal-first": (rho, m_normal, m_tangential..., E).
//
// Nonlinear weights follow Eq. weights literally, omega_m ~ gamma_m / (eps + beta_m)^p,
// with one reciprocal per smoothness window shared by both sides of the face.
// In FP32 eps + beta is kept >= 1e-18 (eps rescaled out of the FP32 denormal
// range: (1e-36)^-2 would overflow); this changes omega only where every
// affected window holds data below ~1e-9, i.e. below FP32 resolution of the
// state.  FP64 uses eps = 1e-36 exactly.
#pragma once
#include <type_traits>
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
    // lower bound of eps + beta in FP32, so that (eps + beta)^-2 stays within range
    static __device__ __forceinline__ float eps_floor() { return 1e-18f; }
    // uncontracted multiply / add (never fused into an FMA, so every kernel rounds alike)
    static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
};

template <>
struct Num<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
    static __device__ __forceinline__ double fmax(double a, double b) { return ::fmax(a, b); }
    static __device__ __forceinline__ double fmin(double a, double b) { return ::fmin(a, b); }
    static __device__ __forceinline__ double eps_floor() { return 0.0; }
    static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
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
    T gwl[R + 1][R + 1];  // gl[m] wl[m][j]: the weighted sum of Eq. weight_sum takes one FMA per m
    T gwr[R + 1][R + 1];  // gr[m] wr[m][j]
    T gsl1[R + 1];        // gl[m] sl1[m]
    T gsr1[R + 1];        // gr[m] sr1[m]
    T Ph[R + 1][(R + 2) / 2];  // P = v / sqrt(lambda) of K_m(sigma), half form, largest lambda first:
                               // even rows symmetric, odd rows skew (K_m is persymmetric)
    T Psum[R + 1];        // sum_j of each full row of P (zero for the skew rows)
    T eps;                // WENO epsilon
    T gamma;              // ratio of specific heats
    int p;                // WENO power, 1 or 2
    int flux;             // face flux: 0 local Lax-Friedrichs, 1 HLLC, 2 HLL
};

// Primitive reference state of the "cell-relative" evaluation (normal-first order).
template <typename T, int NC>
struct PrimRef {
    T rho;            // density of cell s
    T u[NC - 2];      // velocity of cell s
    T p;              // pressure of cell s
    T hp;             // E + p of cell s
    T mn;             // normal momentum rho u_n of cell s (the stored value)
};

// For a primitive perturbation w = V - V_s (V = (rho, u_n, u_t..., p)):
//   cw = U(V) - U(V_s)  (conservative perturbation)
//   G  = F(V) - F(V_s)  (normal-flux perturbation)
// written so that large reference quantities only multiply small ones:
//   g_a = rho u_a - rho_s u_s,a = rho w_a + u_s,a w_rho,  rho = rho_s + w_rho,  u = u_s + w_u
//   k   = rho|u|^2 - rho_s|u_s|^2 = sum_a (g_a u_a + rho_s u_s,a w_a)
//   E'  = w_p/(gamma-1) + k/2
//   G   = (g_n,  g_n u_n + m_s,n w_n + w_p,  g_n u_t + m_s,n w_t,  w_n (E+p)_s + u_n (E' + w_p)).
// Returns false if rho <= 0 or p <= 0 (or NaN); un and cs are the normal velocity and
// the sound speed of the full state.
template <typename T, int NC>
__device__ __forceinline__ bool prim_pert(const PrimRef<T, NC> &r, const T (&w)[NC], T gam, T igm1, T (&G)[NC],
                                          T (&cw)[NC], T &un, T &cs)
{
    constexpr int NV = NC - 2, E = NC - 1;
    const T rho = r.rho + w[0];
    T u[NV], g[NV];
    T k = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        u[a] = r.u[a] + w[1 + a];
        g[a] = fma(rho, w[1 + a], r.u[a] * w[0]);
        k = fma(g[a], u[a], fma(r.rho * r.u[a], w[1 + a], k));
    }
    const T ep = fma(w[E], igm1, T(0.5) * k);
    cw[0] = w[0];
#pragma unroll
    for (int a = 0; a < NV; ++a) cw[1 + a] = g[a];
    cw[E] = ep;
    G[0] = g[0];
    G[1] = fma(g[0], u[0], fma(r.mn, w[1], w[E]));
#pragma unroll
    for (int a = 1; a < NV; ++a) G[1 + a] = fma(g[0], u[a], r.mn * w[1 + a]);
    G[E] = fma(w[1], r.hp, u[0] * (ep + w[E]));
    const T pr = r.p + w[E];
    un = u[0];
    cs = Num<T>::sqrt(Num<T>::fmax(gam * pr * Num<T>::rcp(rho), T(1e-30)));
    return (rho > T(0)) && (pr > T(0));
}

// Roe average of the two cells sharing a face (normal-first conserved uL =
// cell s, uR = cell s+1), the primitive eigen-system at it, and cell s as the
// primitive reference of the cell-relative evaluation:
//   L_V rows: (0, -an, 0, ap), (1, 0, 0, -ie), e_t, (0, an, 0, ap)
//   R_V cols: (1, -cr, 0, c^2), (1, 0, 0, 0),   e_t, (1, cr, 0, c^2)
// with an = rbar/(2c), ap = 1/(2c^2), ie = 1/c^2, cr = c/rbar, rbar = sqrt(rho_L rho_R).
template <typename T, int NC>
struct FaceRoe {
    static constexpr int NV = NC - 2, E = NC - 1;
    T gm1, igm1;
    T vel[NV];        // Roe velocity
    T q2;             // |vel|^2
    T c2, c, ic;      // Roe sound speed squared, sound speed, 1/c
    T rbar, irb;      // sqrt(rho_L rho_R) and its inverse
    T an, ie, ap, cr;
    PrimRef<T, NC> ref;
    T Vs[NC];         // primitive state of cell s
    bool ok;          // rho_L, rho_R, c^2 > 0

    // row kk of L_V applied to a primitive vector
    __device__ __forceinline__ T lrow(int kk, const T *v) const
    {
        if (kk == 0) return fma(ap, v[E], -an * v[1]);
        if (kk == E) return fma(ap, v[E], an * v[1]);
        if (kk == 1) return fma(-ie, v[E], v[0]);
        return v[kk];   // shear: tangential velocity
    }

    // V_j - V_s from the exact conserved difference U_j - U_s by perturbation algebra
    __device__ __forceinline__ void prim_diff(const T (&uj)[NC], const T (&us)[NC], T (&dV)[NC]) const
    {
        T dU[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) dU[a] = uj[a] - us[a];
        const T irj = Num<T>::rcp(uj[0]);
        T k = T(0);
        dV[0] = dU[0];
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            const T du = fma(-ref.u[a], dU[0], dU[1 + a]) * irj;
            dV[1 + a] = du;
            k = fma(uj[1 + a], du, fma(ref.u[a], dU[1 + a], k));
        }
        dV[E] = gm1 * fma(T(-0.5), k, dU[E]);
    }
};

template <typename T, int NC>
__device__ __forceinline__ FaceRoe<T, NC> face_roe(const T (&uL)[NC], const T (&uR)[NC], T gamma)
{
    constexpr int NV = NC - 2, E = NC - 1;
    FaceRoe<T, NC> f;
    f.gm1 = gamma - T(1);
    f.igm1 = Num<T>::rcp(f.gm1);
    const T rL = uL[0], rR = uR[0];
    const T rsL = Num<T>::rsqrt(rL), rsR = Num<T>::rsqrt(rR);
    const T inv = Num<T>::rcp(rL * rsL + rR * rsR);  // 1/(sqrt(rhoL)+sqrt(rhoR))
    const T irL = rsL * rsL;
    T q2 = T(0), mL2 = T(0), mR2 = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        f.vel[a] = fma(uL[1 + a], rsL, uR[1 + a] * rsR) * inv;
        q2 = fma(f.vel[a], f.vel[a], q2);
        mL2 = fma(uL[1 + a], uL[1 + a], mL2);
        mR2 = fma(uR[1 + a], uR[1 + a], mR2);
    }
    const T pL = f.gm1 * fma(T(-0.5) * mL2, irL, uL[E]);
    const T pR = f.gm1 * fma(T(-0.5) * mR2, rsR * rsR, uR[E]);
    const T H = fma(uL[E] + pL, rsL, (uR[E] + pR) * rsR) * inv;
    f.q2 = q2;
    f.c2 = f.gm1 * fma(T(-0.5), q2, H);
    f.ok = (rL > T(0)) && (rR > T(0)) && (f.c2 > T(0));
    f.ic = Num<T>::rsqrt(Num<T>::fmax(f.c2, T(1e-30)));
    f.c = f.c2 * f.ic;
    f.rbar = (rL * rsL) * (rR * rsR);
    f.irb = rsL * rsR;
    f.an = T(0.5) * f.rbar * f.ic;
    f.ie = f.ic * f.ic;
    f.ap = T(0.5) * f.ie;
    f.cr = f.c * f.irb;
    f.ref.rho = rL;
#pragma unroll
    for (int a = 0; a < NV; ++a) f.ref.u[a] = uL[1 + a] * irL;
    f.ref.p = pL;
    f.ref.hp = uL[E] + pL;
    f.ref.mn = uL[1];
    f.Vs[0] = rL;
#pragma unroll
    for (int a = 0; a < NV; ++a) f.Vs[1 + a] = f.ref.u[a];
    f.Vs[E] = pL;
    return f;
}

// (eps + beta)^-p of one smoothness window: beta = sum_h (P_h . (f - shift))^2
// (Eq. beta-eigen) over the window f[w..w+R] of data f_j = f_c + d_j with
// d_R = 0 (relative to the face's cell s).  pf_h = (f_c - shift) sum_j P_hj is
// supplied by the caller (zero for the skew rows, whose sums vanish); rows are
// evaluated in the symmetric/skew half form.
template <typename T, int R, int NS>
__device__ __forceinline__ T beta_weight(const FaceTables<T, R> &tb, const T (&d)[NS], int w, const T (&pf)[R + 1])
{
    constexpr int S = R + 1, HALF = S / 2;
    T ps[HALF > 0 ? HALF : 1], ms[HALF > 0 ? HALF : 1];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const int lo = w + j, hi = w + S - 1 - j;
        ps[j] = lo == R ? d[hi] : (hi == R ? d[lo] : d[lo] + d[hi]);
        ms[j] = lo == R ? -d[hi] : (hi == R ? d[lo] : d[lo] - d[hi]);
    }
    T beta = tb.eps;   // (eps + beta), accumulated from eps
#pragma unroll
    for (int h = 0; h < S; ++h) {
        T dot;
        if (h % 2 == 0) {
            dot = pf[h];
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
    const T x = Num<T>::rcp(Num<T>::fmax(beta, Num<T>::eps_floor()));
    return tb.p == 2 ? Num<T>::mul_rn(x, x) : x;
}

// GP-AO tables (Appendix A) on top of the GP-WENO ones: R = 2 serves AO(2,3),
// R = 3 the recursive AO(3,2,3).  Weights of the full stencil S_R (hi), of
// S_{R-1} (lo, R = 3), of the three 3-point stencils of Eq. cweno_stencil, for
// the left (x* = +1/2) and right (x* = -1/2) states, with their sums minus
// one; half-form factors of K_N(sigma) for N = 2R+1, 2R-1, 3; the linear
// weights of Eq. CWENO-lin.
template <typename T, int R>
struct AoFaceTables : FaceTables<T, R> {
    static constexpr int NH = 2 * R + 1, NL = R > 2 ? 2 * R - 1 : 1;
    T whl[NH], whr[NH], shl, shr;
    T wll[NL], wlr[NL], sll, slr;
    T w3l[3][3], w3r[3][3], s3l[3], s3r[3];
    T Phi[NH][(NH + 1) / 2], Psum_hi[NH];
    T Plo[NL][(NL + 1) / 2], Psum_lo[NL];
    T P3[3][2], Psum3[3];
    T g_hi, g_hi1, ig_hi;   // gamma_HI, 1 - gamma_HI, 1 / gamma_HI
    T g3[3];                // gamma_m = ((1-gHI)(1-gLO)/2, (1-gHI) gLO, (1-gHI)(1-gLO)/2)
};

// (eps + beta)^-p with the FP32 floor on eps + beta (as for GP-WENO)
template <typename T>
__device__ __forceinline__ T inv_pow(T eps, T beta, int p)
{
    const T x = Num<T>::rcp(Num<T>::fmax(Num<T>::add_rn(eps, beta), Num<T>::eps_floor()));
    return p == 2 ? Num<T>::mul_rn(x, x) : x;
}

// sum_h (P_h . (f - shift))^2 over the N-point window f[w..w+N-1] of data
// f_j = f_c + d_j (d_R = 0), P in half form (rows alternately symmetric and
// skew), pf_h = (f_c - shift) sum_j P_hj supplied by the caller.
template <typename T, int N, int R, int NS>
__device__ __forceinline__ T beta_window(const T (&Ph)[N][(N + 1) / 2], const T (&d)[NS], int w, const T (&pf)[N])
{
    constexpr int HALF = N / 2;
    T ps[HALF], ms[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const int lo = w + j, hi = w + N - 1 - j;
        ps[j] = lo == R ? d[hi] : (hi == R ? d[lo] : d[lo] + d[hi]);
        ms[j] = lo == R ? -d[hi] : (hi == R ? d[lo] : d[lo] - d[hi]);
    }
    T beta = T(0);
#pragma unroll
    for (int h = 0; h < N; ++h) {
        T dot;
        if (h % 2 == 0) {
            dot = pf[h];
            if (N % 2 == 1 && w + HALF != R) dot = fma(Ph[h][HALF], d[w + HALF], dot);
#pragma unroll
            for (int j = 0; j < HALF; ++j) dot = fma(Ph[h][j], ps[j], dot);
        } else {
            dot = Ph[h][0] * ms[0];
#pragma unroll
            for (int j = 1; j < HALF; ++j) dot = fma(Ph[h][j], ms[j], dot);
        }
        beta = fma(dot, dot, beta);
    }
    return beta;
}

// GP-AO(R,3) of Eq. GP-AO: the high-order prediction qh, with xh = (eps + beta^R)^-p,
// hybridised with the three 3-point predictions q3 (x3 likewise); weights of Eq.
// nonlin-AO with gamma_HI for the high-order stencil and gamma_m for the small ones.
// The combination's coefficients sum to one, so predictions relative to cell s
// combine to the hybrid relative to cell s.
template <typename T, int R>
__device__ __forceinline__ T ao_hybrid(const AoFaceTables<T, R> &ta, T qh, T xh, const T (&q3)[3], const T (&x3)[3])
{
    const T wh = ta.g_hi * xh;
    T w[3], sum = wh;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        w[m] = ta.g3[m] * x3[m];
        sum += w[m];
    }
    const T inv = Num<T>::rcp(sum);
    const T r = wh * inv * ta.ig_hi;   // omega^R / gamma_HI
    T q = r * qh;
#pragma unroll
    for (int m = 0; m < 3; ++m) q = fma(fma(w[m], inv, -r * ta.g3[m]), q3[m], q);
    return q;
}

// GP-AO prediction of one side of the face, relative to cell s, from the
// characteristic data d (relative to cell s, d_R = 0) and the centre value fc:
// left (RIGHT = false) from the stencil d[0..2R] of cell s at x* = +1/2, right
// from d[1..2R+1] of cell s+1 at x* = -1/2.  beta of each stencil is the
// data-fit term (1/2) f^T K_N(sigma)^-1 f of Eq. log-like, on f (zero mean) or
// on f minus the side's centre value (MEAN).  R = 3 adds the recursive
// hybridisation of AO(3,3) and AO(2,3) (Eqs. recursive-weights, AO-recursive).
template <typename T, int R, int NS, bool RIGHT, bool MEAN>
__device__ __forceinline__ T ao_side(const AoFaceTables<T, R> &ta, const T (&d)[NS], T fc)
{
    constexpr int NH = 2 * R + 1, NL = AoFaceTables<T, R>::NL;
    constexpr int o = RIGHT ? 1 : 0;
    const T shift = MEAN ? (RIGHT ? -d[R + 1] : T(0)) : fc;   // pf_h = Psum_h * shift
    T q3[3], x3[3];
    {
        T pf[3];
#pragma unroll
        for (int h = 0; h < 3; ++h) pf[h] = (h % 2 == 0) ? ta.Psum3[h] * shift : T(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int w0 = o + R - 2 + m;   // Eq. cweno_stencil: cells c-2..c, c-1..c+1, c..c+2
            T q = (RIGHT ? ta.s3r[m] : ta.s3l[m]) * fc;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (w0 + j != R) q = fma(RIGHT ? ta.w3r[m][j] : ta.w3l[m][j], d[w0 + j], q);
            q3[m] = q;
            x3[m] = inv_pow<T>(ta.eps, T(0.5) * beta_window<T, 3, R, NS>(ta.P3, d, w0, pf), ta.p);
        }
    }
    T pfh[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) pfh[h] = (h % 2 == 0) ? ta.Psum_hi[h] * shift : T(0);
    T qh = (RIGHT ? ta.shr : ta.shl) * fc;
#pragma unroll
    for (int j = 0; j < NH; ++j)
        if (o + j != R) qh = fma(RIGHT ? ta.whr[j] : ta.whl[j], d[o + j], qh);
    const T xh = inv_pow<T>(ta.eps, T(0.5) * beta_window<T, NH, R, NS>(ta.Phi, d, o, pfh), ta.p);
    const T q_hi = ao_hybrid<T, R>(ta, qh, xh, q3, x3);
    if constexpr (R == 2) {
        return q_hi;
    } else {
        T pfl[NL];
#pragma unroll
        for (int h = 0; h < NL; ++h) pfl[h] = (h % 2 == 0) ? ta.Psum_lo[h] * shift : T(0);
        T ql = (RIGHT ? ta.slr : ta.sll) * fc;
#pragma unroll
        for (int j = 0; j < NL; ++j)
            if (o + 1 + j != R) ql = fma(RIGHT ? ta.wlr[j] : ta.wll[j], d[o + 1 + j], ql);
        const T xl = inv_pow<T>(ta.eps, T(0.5) * beta_window<T, NL, R, NS>(ta.Plo, d, o + 1, pfl), ta.p);
        const T q_lo = ao_hybrid<T, R>(ta, ql, xl, q3, x3);
        const T vh = ta.g_hi * xh, vl = ta.g_hi1 * xl;
        const T inv = Num<T>::rcp(vh + vl);
        const T rh = vh * inv * ta.ig_hi;   // nu^R' / gamma_HI
        return fma(rh, q_hi, fma(-rh, ta.g_hi1, vl * inv) * q_lo);
    }
}

// Packed FP32: two characteristic fields per instruction (fma/add/mul .f32x2
// of sm_100 and later).  Each lane rounds exactly as the scalar operation.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// beta_weight for two fields at once: (eps + beta)^-p of window d[w..w+R] in each lane.
template <int R, int NS>
__device__ __forceinline__ float2 beta_weight2(const FaceTables<float, R> &tb, const float2 (&d)[NS], int w,
                                               const float2 (&pf)[R + 1])
{
    constexpr int S = R + 1, HALF = S / 2;
    float2 ps[HALF > 0 ? HALF : 1], ms[HALF > 0 ? HALF : 1];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const int lo = w + j, hi = w + S - 1 - j;
        ps[j] = lo == R ? d[hi] : (hi == R ? d[lo] : add2(d[lo], d[hi]));
        ms[j] = lo == R ? mul2(d[hi], f2(-1.0f)) : (hi == R ? d[lo] : sub2(d[lo], d[hi]));
    }
    float2 beta = f2(tb.eps);   // (eps + beta), accumulated from eps
#pragma unroll
    for (int h = 0; h < S; ++h) {
        float2 dot;
        if (h % 2 == 0) {
            dot = pf[h];
            if (S % 2 == 1 && w + HALF != R) dot = fma2(f2(tb.Ph[h][HALF]), d[w + HALF], dot);
#pragma unroll
            for (int j = 0; j < HALF; ++j) dot = fma2(f2(tb.Ph[h][j]), ps[j], dot);
        } else {
            dot = mul2(f2(tb.Ph[h][0]), ms[0]);
#pragma unroll
            for (int j = 1; j < HALF; ++j) dot = fma2(f2(tb.Ph[h][j]), ms[j], dot);
        }
        beta = fma2(dot, dot, beta);
    }
    const float2 x = make_float2(Num<float>::rcp(fmaxf(beta.x, Num<float>::eps_floor())),
                                 Num<float>::rcp(fmaxf(beta.y, Num<float>::eps_floor())));
    return tb.p == 2 ? mul2(x, x) : x;
}

// One face, cell-relative form.  st[0..2R+1] is the normal-first conserved
// stencil; the face s+1/2 lies between st[R] (cell s) and st[R+1] (cell s+1).
// Outputs
//   A = F_{s+1/2} - F(U_s)      (numerical face flux relative to cell s)
//   B = F(U_{s+1}) - F(U_s)     (physical flux difference of the two cells)
// so that the flux jump across cell s, F_{s+1/2} - F_{s-1/2} = A_s - A_{s-1} + B_{s-1},
// is formed from small quantities only.  In real arithmetic this is exactly
// the scheme: characteristic variables of the primitive variables
// V = (rho, u, p) with the eigenvectors of the primitive system at the Roe
// average of cells s, s+1 (Section 6; "FD-Primitive"), GP-WENO states by
// Eqs. candidate_interp, beta-eigen, weights, weight_sum, and the
// Lax-Friedrichs flux.  The rewriting only changes where FP rounding falls:
//   * primitive differences V_j - V_s come from the exact conserved
//     differences U_j - U_s by perturbation algebra, and are projected as
//     d_j = L (V_j - V_s) plus the centre value f_c = L V_s, so
//     q^m = w_m . d_m + f_c sum_j w_mj and P_h . f_m = P_h . d_m + f_c sum_j P_hj;
//   * the left state is V_s + R (q_L - L V_s) and the right state
//     V_{s+1} + R (q_R - L V_{s+1}), using R L = I and sum_m omega_m = 1;
//   * fluxes and conserved states are perturbations about V_s (prim_pert).
// Returns false on a non-physical Roe, left, right or neighbour state.
template <typename T, int NC, int R, bool MEAN = false, bool AO = false>
__device__ __forceinline__ bool face_rel(const T (&st)[2 * R + 2][NC], const FaceTables<T, R> &tb, T (&A)[NC],
                                         T (&B)[NC])
{
    constexpr int NS = 2 * R + 2;
    constexpr int E = NC - 1;
    constexpr int S = R + 1;
    const FaceRoe<T, NC> f = face_roe<T, NC>(st[R], st[R + 1], tb.gamma);
    bool ok = f.ok;
    const T igm1 = f.igm1, c = f.c, c2 = f.c2, cr = f.cr;
    const PrimRef<T, NC> &ref = f.ref;
    const T(&vel)[NC - 2] = f.vel;

    // primitive differences V_j - V_s from the exact conserved differences
    T dV[NS][NC];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (j == R) {
#pragma unroll
            for (int a = 0; a < NC; ++a) dV[j][a] = T(0);
            continue;
        }
        f.prim_diff(st[j], st[R], dV[j]);
    }

    T dqL[NC], dqR[NC];
    // FP32 GP-WENO in 1D and 2D: fields in pairs (0,1), (2,3) through packed
    // instructions, an odd last field (1D) through the scalar loop below.  3D keeps
    // the scalar loop: with five fields the packed form spills registers in the
    // z-marching kernel and measured 3% slower.
    constexpr bool kPacked = std::is_same<T, float>::value && !AO && NC <= 4;
    constexpr int kScalarFrom = kPacked ? (NC / 2) * 2 : 0;
    if constexpr (kPacked) {
#pragma unroll
        for (int k0 = 0; k0 + 1 < NC; k0 += 2) {
            const int k1 = k0 + 1;
            const float2 fc = make_float2(f.lrow(k0, f.Vs), f.lrow(k1, f.Vs));
            float2 d[NS];
#pragma unroll
            for (int j = 0; j < NS; ++j)
                d[j] = (j == R) ? f2(0.0f) : make_float2(f.lrow(k0, dV[j]), f.lrow(k1, dV[j]));
            float2 pfl[S], pfr[S];
#pragma unroll
            for (int h = 0; h < S; ++h) {
                pfl[h] = (h % 2 == 0 && !MEAN) ? mul2(f2(tb.Psum[h]), fc) : f2(0.0f);
                pfr[h] = (h % 2 == 0) ? (MEAN ? mul2(f2(-tb.Psum[h]), d[R + 1]) : pfl[h]) : f2(0.0f);
            }
            float2 numL = f2(0.0f), denL = f2(0.0f), numR = f2(0.0f), denR = f2(0.0f);
            float2 xl = beta_weight2<R, NS>(tb, d, 0, pfl);
#pragma unroll
            for (int m = 0; m <= R; ++m) {
                const float2 xr = beta_weight2<R, NS>(tb, d, m + 1, pfr);
                // gamma_m (candidate_m - centre), with gamma folded into the tables
                float2 sl = mul2(f2(tb.gsl1[m]), fc), sr = mul2(f2(tb.gsr1[m]), fc);
#pragma unroll
                for (int j = 0; j <= R; ++j) {
                    if (m + j != R) sl = fma2(f2(tb.gwl[m][j]), d[m + j], sl);
                    if (1 + m + j != R) sr = fma2(f2(tb.gwr[m][j]), d[1 + m + j], sr);
                }
                numL = fma2(xl, sl, numL);
                denL = fma2(f2(tb.gl[m]), xl, denL);
                numR = fma2(xr, sr, numR);
                denR = fma2(f2(tb.gr[m]), xr, denR);
                if (m < R) xl = MEAN ? beta_weight2<R, NS>(tb, d, m + 1, pfl) : xr;
            }
            const float2 qL = mul2(numL, make_float2(Num<float>::rcp(denL.x), Num<float>::rcp(denL.y)));
            const float2 qR = sub2(mul2(numR, make_float2(Num<float>::rcp(denR.x), Num<float>::rcp(denR.y))), d[R + 1]);
            dqL[k0] = qL.x;
            dqR[k0] = qR.x;
            dqL[k1] = qL.y;
            dqR[k1] = qR.y;
        }
    }
    {
#pragma unroll
    for (int kk = kScalarFrom; kk < NC; ++kk) {
        const T fc = f.lrow(kk, f.Vs);
        T d[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) d[j] = (j == R) ? T(0) : f.lrow(kk, dV[j]);
        if constexpr (AO) {
            // GP-AO predictions relative to cell s (the kernel parameter is AoFaceTables)
            const auto &ta = static_cast<const AoFaceTables<T, R> &>(tb);
            dqL[kk] = ao_side<T, R, NS, false, MEAN>(ta, d, fc);                 // q_L - L V_s
            dqR[kk] = ao_side<T, R, NS, true, MEAN>(ta, d, fc) - d[R + 1];      // q_R - L V_{s+1}
        } else {
            // zero mean: both sides shift by f_c, so the right side's window m is the
            // left side's window m+1 and the R+2 windows are shared.  Mean f_centre:
            // the left side's centre is cell s (no shift), the right side's is cell
            // s+1 (shift by d_{R+1}), and the 2R+2 windows are separate.
            T pfl[S], pfr[S];
#pragma unroll
            for (int h = 0; h < S; ++h) {
                pfl[h] = (h % 2 == 0 && !MEAN) ? tb.Psum[h] * fc : T(0);
                pfr[h] = (h % 2 == 0) ? (MEAN ? -tb.Psum[h] * d[R + 1] : pfl[h]) : T(0);
            }
            // --- candidates relative to the centre cells and nonlinear weights ---
            // omega_m ~ gamma_m (eps + beta_m)^-p  (Eq. weights); sum_m omega_m = 1 is used exactly.
            T numL = T(0), denL = T(0), numR = T(0), denR = T(0);
            T xl = beta_weight<T, R, NS>(tb, d, 0, pfl);
#pragma unroll
            for (int m = 0; m <= R; ++m) {
                const T xr = beta_weight<T, R, NS>(tb, d, m + 1, pfr);
                T sl = tb.gsl1[m] * fc, sr = tb.gsr1[m] * fc;   // gamma_m (candidate_m - centre)
#pragma unroll
                for (int j = 0; j <= R; ++j) {
                    if (m + j != R) sl = fma(tb.gwl[m][j], d[m + j], sl);
                    if (1 + m + j != R) sr = fma(tb.gwr[m][j], d[1 + m + j], sr);
                }
                numL = fma(xl, sl, numL);
                denL = fma(tb.gl[m], xl, denL);
                numR = fma(xr, sr, numR);
                denR = fma(tb.gr[m], xr, denR);
                if (m < R) xl = MEAN ? beta_weight<T, R, NS>(tb, d, m + 1, pfl) : xr;
            }
            dqL[kk] = numL * Num<T>::rcp(denL);              // q_L - L V_s
            dqR[kk] = numR * Num<T>::rcp(denR) - d[R + 1];   // q_R - L V_{s+1}
        }
    }
    }

    // --- back-projection: primitive states relative to cell s -------------
    T wL[NC], wR[NC];
    wL[0] = dqL[0] + dqL[1] + dqL[E];
    wR[0] = dV[R + 1][0] + (dqR[0] + dqR[1] + dqR[E]);
    wL[1] = cr * (dqL[E] - dqL[0]);
    wR[1] = fma(cr, dqR[E] - dqR[0], dV[R + 1][1]);
#pragma unroll
    for (int a = 2; a < E; ++a) {
        wL[a] = dqL[a];
        wR[a] = dV[R + 1][a] + dqR[a];
    }
    wL[E] = c2 * (dqL[0] + dqL[E]);
    wR[E] = fma(c2, dqR[0] + dqR[E], dV[R + 1][E]);

    // --- face flux relative to F(U_s), and F(U_{s+1}) - F(U_s) ---------------
    T GL[NC], GR[NC], cL[NC], cR[NC], cB[NC], uL, uR, aL, aR, uB, aB;
    ok = prim_pert<T, NC>(ref, wL, tb.gamma, igm1, GL, cL, uL, aL) && ok;
    ok = prim_pert<T, NC>(ref, wR, tb.gamma, igm1, GR, cR, uR, aR) && ok;
    T dn[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) dn[a] = dV[R + 1][a];
    ok = prim_pert<T, NC>(ref, dn, tb.gamma, igm1, B, cB, uB, aB) && ok;
    if (tb.flux == 1) {
        // HLLC with Einfeldt speeds from the Roe average.  The contact speed enters only
        // through S* - u_K = (dp - rho_K' (S_K' - u_K') du) / D (K' the other side), formed
        // from the small differences dp = p_R - p_L, du = u_R - u_L, so the star states
        // U*_K - U_K stay accurate increments.
        const T rhoL = ref.rho + wL[0], rhoR = ref.rho + wR[0];
        const T pLf = ref.p + wL[E], pRf = ref.p + wR[E];
        const T SL = Num<T>::fmin(uL - aL, vel[0] - c), SR = Num<T>::fmax(uR + aR, vel[0] + c);
        const T mL = rhoL * (SL - uL), mR = rhoR * (SR - uR);
        const T iD = Num<T>::rcp(mL - mR);
        const T dp = wR[E] - wL[E], du = wR[1] - wL[1];
        const T sL = (dp - mR * du) * iD;   // S* - u_L
        const T sR = (dp - mL * du) * iD;   // S* - u_R
        const T Ss = uL + sL;
        const T Es = ref.hp - ref.p;
        auto star = [&](const T (&w)[NC], const T (&cw)[NC], T rho, T pK, T mK, T SK, T sK, T (&dU)[NC]) {
            // U*_K - U_K with chi = rho_K (S_K - u_K) / (S_K - S*), chi - 1 = (S* - u_K) / (S_K - S*)
            const T q = Num<T>::rcp(mK * Num<T>::rcp(rho) - sK);   // 1 / (S_K - S*)
            const T chi1 = sK * q;
            dU[0] = rho * chi1;
            dU[1] = rho * fma(chi1, Ss, sK);
#pragma unroll
            for (int a = 2; a < E; ++a) dU[a] = rho * (ref.u[a - 1] + w[a]) * chi1;
            const T EK = Es + cw[E];
            // chi rho_K (S* - u_K)(S* + p_K / (rho_K (S_K - u_K))), with chi rho_K = m_K q
            dU[E] = fma(chi1, EK, mK * q * sK * (Ss + pK * Num<T>::rcp(mK)));
        };
        T dUL[NC], dUR[NC];
        star(wL, cL, rhoL, pLf, mL, SL, sL, dUL);
        star(wR, cR, rhoR, pRf, mR, SR, sR, dUR);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            T f;
            if (SL >= T(0)) f = GL[a];
            else if (SR <= T(0)) f = GR[a];
            else if (Ss >= T(0)) f = fma(SL, dUL[a], GL[a]);
            else f = fma(SR, dUR[a], GR[a]);
            A[a] = f;
        }
    } else if (tb.flux == 2) {
        // HLL with the same Einfeldt speeds: F_L if S_L >= 0, F_R if S_R <= 0, else
        // (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L); relative to F(U_s)
        // the flux terms keep that form with G_K = F_K - F(U_s) and c_K = U_K - U_s.
        const T SL = Num<T>::fmin(uL - aL, vel[0] - c), SR = Num<T>::fmax(uR + aR, vel[0] + c);
        const T iS = Num<T>::rcp(SR - SL);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            T f;
            if (SL >= T(0)) f = GL[a];
            else if (SR <= T(0)) f = GR[a];
            else f = (fma(SR, GL[a], -SL * GR[a]) + SL * SR * (cR[a] - cL[a])) * iS;
            A[a] = f;
        }
    } else {
        const T alpha = Num<T>::fmax(Num<T>::fabs(uL) + aL, Num<T>::fabs(uR) + aR);
#pragma unroll
        for (int a = 0; a < NC; ++a) A[a] = T(0.5) * ((GL[a] + GR[a]) - alpha * (cR[a] - cL[a]));
    }
    return ok;
}

// One face of the FD-Flux form (Section 2), cell-relative; outputs as face_rel:
//   A = f^_{s+1/2} - F(U_s),  B = F(U_{s+1}) - F(U_s).
// The point fluxes are cell averages of the function whose face values are
// the numerical fluxes (Eqs. prim_F, design).  They are split by local
// Lax-Friedrichs, F+- = (F +- alpha U)/2 with alpha the largest |u_n| + c over
// the 2R+2 stencil cells, projected on the characteristic fields of the
// conservative Jacobian at the Roe average, l(X) = L_V (dV/dU) X with dV/dU
// taken at (rbar, vel, c) (the conservative Jacobian depends on the state only
// through vel and H, so these are its left eigenvectors up to row scaling),
// reconstructed by GP-WENO -- F+ on the stencil of cell s at x* = +1/2, F- on
// that of cell s+1 at x* = -1/2, the tables holding reconstruction weights --
// and projected back with (dU/dV) R_V.  Everything is relative to cell s:
// with d+-_j = (l(F_j - F_s) +- alpha l(U_j - U_s)) / 2 and g+-_s the cell-s
// values, each reconstructed part minus g+-_s is
// sum_m omega_m (w_m . d_m + (sum_j w_mj - 1) g+-_s), and g+_s + g-_s = l(F_s)
// projects back to F(U_s).  Returns false on a non-physical state.
template <typename T, int NC, int R, bool MEAN = false>
__device__ __forceinline__ bool face_fdf(const T (&st)[2 * R + 2][NC], const FaceTables<T, R> &tb, T (&A)[NC],
                                         T (&B)[NC])
{
    constexpr int NS = 2 * R + 2, E = NC - 1, NV = NC - 2, S = R + 1;
    const FaceRoe<T, NC> f = face_roe<T, NC>(st[R], st[R + 1], tb.gamma);
    bool ok = f.ok;

    // splitting speed: the largest |u_n| + c over the stencil
    T alpha = T(0);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const T ir = Num<T>::rcp(st[j][0]);
        T m2 = T(0);
#pragma unroll
        for (int a = 0; a < NV; ++a) m2 = fma(st[j][1 + a], st[j][1 + a], m2);
        const T pj = f.gm1 * fma(T(-0.5) * m2, ir, st[j][E]);
        ok = ok && (st[j][0] > T(0)) && (pj > T(0));
        alpha = Num<T>::fmax(alpha, Num<T>::fabs(st[j][1] * ir) +
                                        Num<T>::sqrt(Num<T>::fmax(tb.gamma * pj * ir, T(0))));
    }
    // dV/dU at the Roe state applied to a conserved vector
    auto jac = [&](const T (&X)[NC], T (&Y)[NC]) {
        Y[0] = X[0];
        T k = T(0);
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            Y[1 + a] = fma(-f.vel[a], X[0], X[1 + a]) * f.irb;
            k = fma(f.vel[a], X[1 + a], k);
        }
        Y[E] = f.gm1 * (fma(T(0.5) * f.q2, X[0], X[E]) - k);
    };
    // cell s: U_s and F(U_s)
    T Fs[NC];
    Fs[0] = st[R][1];
    Fs[1] = fma(st[R][1], f.ref.u[0], f.ref.p);
#pragma unroll
    for (int a = 1; a < NV; ++a) Fs[1 + a] = st[R][1] * f.ref.u[a];
    Fs[E] = f.ref.u[0] * f.ref.hp;
    T JUs[NC], JFs[NC];
    jac(st[R], JUs);
    jac(Fs, JFs);

    // characteristic increments of the split fluxes, relative to cell s
    T dp[NC][NS], dm[NC][NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (j == R) {
#pragma unroll
            for (int k = 0; k < NC; ++k) dp[k][j] = dm[k][j] = T(0);
            continue;
        }
        T dV[NC], G[NC], cw[NC], un, cs;
        f.prim_diff(st[j], st[R], dV);
        ok = prim_pert<T, NC>(f.ref, dV, tb.gamma, f.igm1, G, cw, un, cs) && ok;
        if (j == R + 1) {
#pragma unroll
            for (int a = 0; a < NC; ++a) B[a] = G[a];
        }
        T dU[NC], JdU[NC], JG[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) dU[a] = st[j][a] - st[R][a];
        jac(dU, JdU);
        jac(G, JG);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const T lg = f.lrow(k, JG), lv = f.lrow(k, JdU);
            dp[k][j] = T(0.5) * fma(alpha, lv, lg);
            dm[k][j] = T(0.5) * fma(-alpha, lv, lg);
        }
    }

    T dq[NC];
    // FP32 in 1D and 2D: fields in pairs through packed instructions (as in face_rel);
    // 3D and an odd last field take the scalar loop.
    constexpr bool kPacked = std::is_same<T, float>::value && NC <= 4;
    constexpr int kScalarFrom = kPacked ? (NC / 2) * 2 : 0;
    if constexpr (kPacked) {
#pragma unroll
        for (int k0 = 0; k0 + 1 < NC; k0 += 2) {
            const int k1 = k0 + 1;
            const float2 lgs = make_float2(f.lrow(k0, JFs), f.lrow(k1, JFs));
            const float2 lvs = make_float2(f.lrow(k0, JUs), f.lrow(k1, JUs));
            const float2 fcp = mul2(f2(0.5f), fma2(f2(alpha), lvs, lgs));
            const float2 fcm = mul2(f2(0.5f), fma2(f2(-alpha), lvs, lgs));
            float2 p2[NS], m2[NS];
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                p2[j] = make_float2(dp[k0][j], dp[k1][j]);
                m2[j] = make_float2(dm[k0][j], dm[k1][j]);
            }
            float2 pfl[S], pfr[S];
#pragma unroll
            for (int h = 0; h < S; ++h) {
                pfl[h] = (h % 2 == 0 && !MEAN) ? mul2(f2(tb.Psum[h]), fcp) : f2(0.0f);
                pfr[h] = (h % 2 == 0) ? (MEAN ? mul2(f2(-tb.Psum[h]), m2[R + 1]) : mul2(f2(tb.Psum[h]), fcm))
                                      : f2(0.0f);
            }
            float2 numL = f2(0.0f), denL = f2(0.0f), numR = f2(0.0f), denR = f2(0.0f);
#pragma unroll
            for (int m = 0; m <= R; ++m) {
                const float2 xl = beta_weight2<R, NS>(tb, p2, m, pfl);
                const float2 xr = beta_weight2<R, NS>(tb, m2, m + 1, pfr);
                float2 sl = mul2(f2(tb.gsl1[m]), fcp), sr = mul2(f2(tb.gsr1[m]), fcm);
#pragma unroll
                for (int j = 0; j <= R; ++j) {
                    if (m + j != R) sl = fma2(f2(tb.gwl[m][j]), p2[m + j], sl);
                    if (1 + m + j != R) sr = fma2(f2(tb.gwr[m][j]), m2[1 + m + j], sr);
                }
                numL = fma2(xl, sl, numL);
                denL = fma2(f2(tb.gl[m]), xl, denL);
                numR = fma2(xr, sr, numR);
                denR = fma2(f2(tb.gr[m]), xr, denR);
            }
            const float2 q = fma2(numL, make_float2(Num<float>::rcp(denL.x), Num<float>::rcp(denL.y)),
                                  mul2(numR, make_float2(Num<float>::rcp(denR.x), Num<float>::rcp(denR.y))));
            dq[k0] = q.x;
            dq[k1] = q.y;
        }
    }
#pragma unroll
    for (int kk = kScalarFrom; kk < NC; ++kk) {
        const T lgs = f.lrow(kk, JFs), lvs = f.lrow(kk, JUs);
        const T fcp = T(0.5) * fma(alpha, lvs, lgs), fcm = T(0.5) * fma(-alpha, lvs, lgs);
        // zero mean: shifts g+_s and g-_s; mean: centres cell s (left) and s+1 (right)
        T pfl[S], pfr[S];
#pragma unroll
        for (int h = 0; h < S; ++h) {
            pfl[h] = (h % 2 == 0 && !MEAN) ? tb.Psum[h] * fcp : T(0);
            pfr[h] = (h % 2 == 0) ? (MEAN ? -tb.Psum[h] * dm[kk][R + 1] : tb.Psum[h] * fcm) : T(0);
        }
        T numL = T(0), denL = T(0), numR = T(0), denR = T(0);
#pragma unroll
        for (int m = 0; m <= R; ++m) {
            const T xl = beta_weight<T, R, NS>(tb, dp[kk], m, pfl);
            const T xr = beta_weight<T, R, NS>(tb, dm[kk], m + 1, pfr);
            T sl = tb.gsl1[m] * fcp, sr = tb.gsr1[m] * fcm;
#pragma unroll
            for (int j = 0; j <= R; ++j) {
                if (m + j != R) sl = fma(tb.gwl[m][j], dp[kk][m + j], sl);
                if (1 + m + j != R) sr = fma(tb.gwr[m][j], dm[kk][1 + m + j], sr);
            }
            numL = fma(xl, sl, numL);
            denL = fma(tb.gl[m], xl, denL);
            numR = fma(xr, sr, numR);
            denR = fma(tb.gr[m], xr, denR);
        }
        dq[kk] = fma(numL, Num<T>::rcp(denL), numR * Num<T>::rcp(denR));
    }

    // back-projection A = (dU/dV) R_V dq at the Roe state
    T w[NC];
    w[0] = dq[0] + dq[1] + dq[E];
    w[1] = f.cr * (dq[E] - dq[0]);
#pragma unroll
    for (int a = 2; a < E; ++a) w[a] = dq[a];
    w[E] = f.c2 * (dq[0] + dq[E]);
    A[0] = w[0];
    T ke = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        A[1 + a] = fma(f.vel[a], w[0], f.rbar * w[1 + a]);
        ke = fma(f.vel[a], w[1 + a], ke);
    }
    A[E] = fma(T(0.5) * f.q2, w[0], fma(f.rbar, ke, w[E] * f.igm1));
    return ok;
}

// Scheme variants chosen at compile time: bit 0 the non-zero-mean smoothness
// indicators, bit 1 the FD-Flux form, bit 2 GP-AO; bit 3 is not a scheme change
// but a grid with an external (halo) side, whose loaders read ghost layers from
// halo buffers -- a separate instantiation so that the loaders of the others stay
// as they are.
constexpr int kVarMean = 1, kVarFdFlux = 2, kVarAo = 4, kVarSlab = 8;

// Kernel parameter type of a variant's tables.
template <typename T, int R, int VAR>
using TablesFor = typename std::conditional<(VAR & kVarAo) != 0, AoFaceTables<T, R>, FaceTables<T, R>>::type;

template <typename T, int NC, int R, int VAR>
__device__ __forceinline__ bool face_eval(const T (&st)[2 * R + 2][NC], const FaceTables<T, R> &tb, T (&A)[NC],
                                          T (&B)[NC])
{
    if constexpr ((VAR & kVarFdFlux) != 0) return face_fdf<T, NC, R, (VAR & kVarMean) != 0>(st, tb, A, B);
    else return face_rel<T, NC, R, (VAR & kVarMean) != 0, (VAR & kVarAo) != 0>(st, tb, A, B);
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

// Flux difference across a cell from the five face-flux differences around it:
// corrected in the FD-Prim form; in the FD-Flux form the reconstructed flux is
// itself the numerical flux (Eq. design), so only the centre one is used.
template <typename T, int VAR>
__device__ __forceinline__ T flux_divergence(T d0, T d1, T d2, T d3, T d4)
{
    if constexpr ((VAR & kVarFdFlux) != 0) return d2;
    else return corrected_divergence<T>(d0, d1, d2, d3, d4);
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
