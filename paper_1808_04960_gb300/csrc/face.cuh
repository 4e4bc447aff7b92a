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
    T wl[R + 1][R + 1];   // sub-stencil weights, left state
    T wr[R + 1][R + 1];   // sub-stencil weights, right state
    T gl[R + 1];          // linear weights, left state
    T gr[R + 1];          // linear weights, right state
    T Ph[R + 1][(R + 2) / 2];  // P_h = v_h / sqrt(lambda_h) of K_m(sigma), half form, largest lambda first:
                               // even rows symmetric, odd rows skew (K_m is persymmetric)
    T eps;                // WENO epsilon
    T gamma;              // ratio of specific heats
    int p;                // WENO power, 1 or 2
};

// Nonlinear GP-WENO combination for one side: candidates q[m], beta windows b[m]
// (already eps + beta), linear weights g[m].
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

// Flux of a normal-first state along its normal; returns false if the state
// is not physical (rho <= 0, p <= 0 or NaN).  Also returns |u_n| + c.
template <typename T, int NC>
__device__ __forceinline__ bool euler_flux(const T (&u)[NC], T gam, T (&f)[NC], T &speed)
{
    T rho = u[0];
    T ir = Num<T>::rcp(rho);
    T un = u[1] * ir;
    T m2 = u[1] * u[1];
#pragma unroll
    for (int a = 2; a < NC - 1; ++a) m2 = fma(u[a], u[a], m2);
    T pr = (gam - T(1)) * (u[NC - 1] - T(0.5) * m2 * ir);
    f[0] = u[1];
    f[1] = fma(u[1], un, pr);
#pragma unroll
    for (int a = 2; a < NC - 1; ++a) f[a] = u[a] * un;
    f[NC - 1] = un * (u[NC - 1] + pr);
    T c2 = gam * pr * ir;
    speed = Num<T>::fabs(un) + Num<T>::sqrt(Num<T>::fmax(c2, T(0)));
    return (rho > T(0)) && (pr > T(0));
}

// Face flux from a normal-first stencil st[0..2R+1]; the face lies between
// st[R] and st[R+1].  Returns false on a non-physical Roe, left or right state.
template <typename T, int NC, int R>
__device__ __forceinline__ bool face_flux(const T (&st)[2 * R + 2][NC], const FaceTables<T, R> &tb, T (&F)[NC])
{
    constexpr int NS = 2 * R + 2;
    constexpr int E = NC - 1;
    constexpr int NV = NC - 2;  // velocity components
    const T gm1 = tb.gamma - T(1);

    // --- Roe average of the two cells sharing the face -------------------
    const T rL = st[R][0], rR = st[R + 1][0];
    const T rsL = Num<T>::rsqrt(rL), rsR = Num<T>::rsqrt(rR);
    const T inv = Num<T>::rcp(rL * rsL + rR * rsR);  // 1/(sqrt(rhoL)+sqrt(rhoR))
    T vel[NV];
    T q2 = T(0);
    T mL2 = T(0), mR2 = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        vel[a] = fma(st[R][1 + a], rsL, st[R + 1][1 + a] * rsR) * inv;
        q2 = fma(vel[a], vel[a], q2);
        mL2 = fma(st[R][1 + a], st[R][1 + a], mL2);
        mR2 = fma(st[R + 1][1 + a], st[R + 1][1 + a], mR2);
    }
    const T pL = gm1 * (st[R][E] - T(0.5) * mL2 * Num<T>::rcp(rL));
    const T pR = gm1 * (st[R + 1][E] - T(0.5) * mR2 * Num<T>::rcp(rR));
    const T H = fma(st[R][E] + pL, rsL, (st[R + 1][E] + pR) * rsR) * inv;
    const T c2 = gm1 * (H - T(0.5) * q2);
    bool ok = (rL > T(0)) && (rR > T(0)) && (c2 > T(0));
    const T ic = Num<T>::rsqrt(Num<T>::fmax(c2, T(1e-30)));
    const T c = c2 * ic;
    const T un = vel[0];
    const T b1 = gm1 * ic * ic;
    const T b2 = T(0.5) * q2 * b1;
    const T hb1 = T(0.5) * b1;

    // characteristic states (left / right prediction) per field
    T qL[NC], qR[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        // --- projection of the stencil on field k (row k of L) -----------
        T f[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const T *u = st[j];
            T v;
            if (k == 0 || k == E) {
                // acoustic rows: 1/2 (b2 +- un/c, -b1 un -+ 1/c, -b1 v_t, b1)
                const T sgn = (k == 0) ? T(1) : T(-1);
                T acc = fma(hb1, u[E], T(0.5) * (b2 + sgn * un * ic) * u[0]);
                acc = fma(T(-0.5) * (b1 * un + sgn * ic), u[1], acc);
#pragma unroll
                for (int a = 1; a < NV; ++a) acc = fma(-hb1 * vel[a], u[1 + a], acc);
                v = acc;
            } else if (k == 1) {
                // entropy row: (1 - b2, b1 u_a..., -b1)
                T acc = fma(-b1, u[E], (T(1) - b2) * u[0]);
#pragma unroll
                for (int a = 0; a < NV; ++a) acc = fma(b1 * vel[a], u[1 + a], acc);
                v = acc;
            } else {
                // shear row of tangential velocity k-1: (-v_t, ..., 1, ...)
                v = fma(-vel[k - 1], u[0], u[k]);
            }
            f[j] = v;
        }
        // --- smoothness indicators on the R+2 windows f[w..w+R] ----------
        // beta = sum_h (P_h . f)^2 with P_h symmetric or skew: pair f_j with
        // f_{S-1-j} once, then each dot product takes half the multiplies.
        constexpr int S = R + 1, HALF = S / 2;
        T b[R + 2];
#pragma unroll
        for (int w = 0; w < R + 2; ++w) {
            T ps[HALF > 0 ? HALF : 1], ms[HALF > 0 ? HALF : 1];
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                ps[j] = f[w + j] + f[w + S - 1 - j];
                ms[j] = f[w + j] - f[w + S - 1 - j];
            }
            T beta = T(0);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                T d;
                if (k % 2 == 0) {
                    if (S % 2 == 1) {
                        d = tb.Ph[k][HALF] * f[w + HALF];
#pragma unroll
                        for (int j = 0; j < HALF; ++j) d = fma(tb.Ph[k][j], ps[j], d);
                    } else {
                        d = tb.Ph[k][0] * ps[0];
#pragma unroll
                        for (int j = 1; j < HALF; ++j) d = fma(tb.Ph[k][j], ps[j], d);
                    }
                } else {
                    d = tb.Ph[k][0] * ms[0];
#pragma unroll
                    for (int j = 1; j < HALF; ++j) d = fma(tb.Ph[k][j], ms[j], d);
                }
                beta = fma(d, d, beta);
            }
            b[w] = tb.eps + beta;
        }
        // --- candidates and nonlinear combination, both sides ------------
        T cl[R + 1], cr[R + 1], bl[R + 1], br[R + 1];
#pragma unroll
        for (int m = 0; m <= R; ++m) {
            T sl = T(0), sr = T(0);
#pragma unroll
            for (int j = 0; j <= R; ++j) {
                sl = fma(tb.wl[m][j], f[m + j], sl);
                sr = fma(tb.wr[m][j], f[1 + m + j], sr);
            }
            cl[m] = sl;
            cr[m] = sr;
            bl[m] = b[m];
            br[m] = b[m + 1];
        }
        qL[k] = weno_combine<T, R>(cl, bl, tb.gl, tb.p);
        qR[k] = weno_combine<T, R>(cr, br, tb.gr, tb.p);
    }

    // --- back-projection U = R q (columns of R written out) --------------
    T uL[NC], uR[NC];
    {
        const T hL = qL[0] + qL[1] + qL[E], hR = qR[0] + qR[1] + qR[E];
        uL[0] = hL;
        uR[0] = hR;
        uL[1] = fma(un, hL, c * (qL[E] - qL[0]));
        uR[1] = fma(un, hR, c * (qR[E] - qR[0]));
        T eL = fma(H, qL[0] + qL[E], fma(T(0.5) * q2, qL[1], un * c * (qL[E] - qL[0])));
        T eR = fma(H, qR[0] + qR[E], fma(T(0.5) * q2, qR[1], un * c * (qR[E] - qR[0])));
#pragma unroll
        for (int a = 1; a < NV; ++a) {
            uL[1 + a] = fma(vel[a], hL, qL[1 + a]);
            uR[1 + a] = fma(vel[a], hR, qR[1 + a]);
            eL = fma(vel[a], qL[1 + a], eL);
            eR = fma(vel[a], qR[1 + a], eR);
        }
        uL[E] = eL;
        uR[E] = eR;
    }

    // --- local Lax-Friedrichs flux ----------------------------------------
    T fL[NC], fR[NC], sL, sR;
    ok = euler_flux<T, NC>(uL, tb.gamma, fL, sL) && ok;
    ok = euler_flux<T, NC>(uR, tb.gamma, fR, sR) && ok;
    const T alpha = Num<T>::fmax(sL, sR);
#pragma unroll
    for (int a = 0; a < NC; ++a) F[a] = T(0.5) * ((fL[a] + fR[a]) - alpha * (uR[a] - uL[a]));
    return ok;
}

// Corrected numerical flux from five consecutive face fluxes F_{s-2..s+2}
// (Eqs. numFlux_cor, FD-ders; alpha = -1/24, beta = 3/640; the dx^2, dx^4
// factors cancel against the finite-difference denominators).
template <typename T>
__device__ __forceinline__ T corrected(T fm2, T fm1, T f0, T fp1, T fp2)
{
    const T d2 = fm1 - T(2) * f0 + fp1;
    const T d4 = fm2 - T(4) * (fm1 + fp1) + T(6) * f0 + fp2;
    return f0 + T(-1.0 / 24.0) * d2 + T(3.0 / 640.0) * d4;
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
