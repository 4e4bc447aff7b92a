// Fused GP-WENO stage kernels: RHS (Eq. disc_fd with the corrected fluxes of
// Eq. numFlux_cor) fused with the SSP-RK3 stage combination.
//
// 2D design ("column-strip marching").  A CTA owns a strip of W <= NT-5
// columns and a segment of rows [y0, y1).  It walks the y-faces s+1/2 from
// s = y0-3 to y1+1 once each:
//   * each thread owns one column and keeps the last five y-face fluxes of
//     that column in registers, so every y-face is evaluated exactly once and
//     the y-correction (five neighbouring faces) needs no shared memory;
//   * the rows of the strip (with R+3 ghost columns per side, boundary
//     conditions applied on load) stream through a small shared-memory ring
//     filled by cp.async one row ahead of use;
//   * for the output row r = s-2, the W+5 x-faces of that row are evaluated
//     from the ring (one per thread), staged in shared memory, corrected,
//     differenced, and combined with the y-part and the RK stage update;
//     the result is stored once (coalesced).
// Per output row a CTA evaluates W y-faces and W+5 x-faces, so the only
// redundant face work is 5 x-faces per row per strip and 5 warm-up y-faces
// per column per segment.
//
// HBM traffic per cell and stage: the stage input state once (ring rows are
// read once per strip; ghost columns come from L2), U^n once for stages 2-3,
// the output once.
#pragma once
#include "face.cuh"

namespace gpweno {

template <typename T>
struct StageArgs {
    const T *U;                // stage input (stencil) state, SoA [nc][nz][ny][nx]
    const T *U0;               // U^n for the stage combination (unused if a0 == 0 or mode == 0)
    T *out;                    // result
    int n[3];                  // cells per dimension (x, y, z)
    int per[3];                // periodic flag per dimension
    T idx[3];                  // 1/dx per dimension
    T a0, b;                   // stage: out = a0 U0 + b (U + dt L(U))
    int mode;                  // 0: out = L(U); 1: stage combination
    const double *dt_dev;      // device dt (or null: use dt)
    double dt;
    unsigned long long *rate;  // if non-null: atomic max of (|u_d| + c)/dx_d of the result (double bits)
    int *flags;                // bit 0: non-physical state met
    int W, nstrips, H, nseg;   // schedule: strip width, #strips, segment height, #segments
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(sizeof(T)));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Ring geometry of the 2D kernel for radius R and block size NT.
template <int R, int NT>
struct Ring2D {
    static constexpr int G = R + 3;                      // ghost layers
    static constexpr int LOW = R > 2 ? R : 2;            // rows below s still in use
    static constexpr int NEEDED = LOW + R + 3;           // rows s-LOW .. s+R+2 (one prefetched)
    static constexpr int ROWS = NEEDED <= 8 ? 8 : 16;    // power of two: slot = row & (ROWS-1)
    static constexpr int STRIDE = NT - 5 + 2 * G;        // elements per ring row and component
    static constexpr int WMAX = NT - 5;
    static __device__ __forceinline__ int slot(int g) { return g & (ROWS - 1); }
};

template <typename T, int R, int NT>
constexpr size_t stage2d_smem_bytes()
{
    using RG = Ring2D<R, NT>;
    return sizeof(T) * (size_t)(RG::ROWS * 4 * RG::STRIDE + 4 * NT);
}

// Rate (|u_d| + c) / dx_d of a natural-order 2D state.
template <typename T>
__device__ __forceinline__ void rates2d(const T (&u)[4], T gam, const T (&idx)[3], T &rx, T &ry)
{
    T ir = Num<T>::rcp(u[0]);
    T vx = u[1] * ir, vy = u[2] * ir;
    T pr = (gam - T(1)) * (u[3] - T(0.5) * (u[1] * vx + u[2] * vy));
    T c = Num<T>::sqrt(Num<T>::fmax(gam * pr * ir, T(0)));
    rx = (Num<T>::fabs(vx) + c) * idx[0];
    ry = (Num<T>::fabs(vy) + c) * idx[1];
}

// One segment: rows [y0, y1) of strip `strip`.
template <typename T, int R, int NT>
__device__ __forceinline__ void stage2d_segment(const StageArgs<T> &a, const FaceTables<T, R> &tb, int strip, int y0,
                                                int y1, T *smem, T dt, T &rmx, T &rmy, bool &ok)
{
    using RG = Ring2D<R, NT>;
    constexpr int G = RG::G, ROWS = RG::ROWS, STRIDE = RG::STRIDE;
    constexpr int NC = 4;
    constexpr int NS = 2 * R + 2;
    T *ring = smem;                              // [ROWS][NC][STRIDE]
    T *Fx = smem + ROWS * NC * STRIDE;           // [NC][NT]
    const int tid = threadIdx.x;
    const int nx = a.n[0], ny = a.n[1];
    const long plane = (long)nx * ny;
    const int x0 = strip * a.W;
    const int Wc = min(a.W, nx - x0);
    const int s_begin = y0 - 3, s_end = y1 + 1;
    const int rowlen = Wc + 2 * G;
    const T idx[3] = {a.idx[0], a.idx[1], a.idx[2]};

    auto load_row = [&](int g) {
        const int gy = bc_map(g, ny, a.per[1]);
        T *dst = ring + RG::slot(g) * (NC * STRIDE);
        const T *src = a.U + (long)gy * nx;
        for (int col = tid; col < rowlen; col += NT) {
            const int gx = bc_map(x0 - G + col, nx, a.per[0]);
#pragma unroll
            for (int c = 0; c < NC; ++c) cp_async_elem(dst + c * STRIDE + col, src + c * plane + gx);
        }
    };

    // prologue: rows needed by the first y-face
    for (int g = s_begin - R; g <= s_begin + 1 + R; ++g) load_row(g);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    T Fy[5][NC];
    T fy_prev[NC];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) Fy[k][c] = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) fy_prev[c] = T(0);

    for (int s = s_begin; s <= s_end; ++s) {
        if (s < s_end) load_row(s + 2 + R);
        cp_async_commit();
        const int r = s - 2;
        const bool out_row = r >= y0;
        const bool col_ok = tid < Wc;

        // U^n of this thread's output cell, in flight during the face work
        T u0[NC];
        const bool need_u0 = out_row && col_ok && a.mode == 1 && a.a0 != T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) u0[c] = need_u0 ? a.U0[c * plane + (long)r * nx + x0 + tid] : T(0);

        // ---- y-face s+1/2 of column tid --------------------------------
        if (col_ok) {
            T st[NS][NC];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const T *row = ring + RG::slot(s - R + q) * (NC * STRIDE) + G + tid;
                st[q][0] = row[0];
                st[q][1] = row[2 * STRIDE];   // normal momentum: rho v
                st[q][2] = row[1 * STRIDE];   // tangential: rho u
                st[q][3] = row[3 * STRIDE];
            }
            T F[NC];
            ok = face_flux<T, NC, R>(st, tb, F) && ok;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) Fy[k][c] = Fy[k + 1][c];
            Fy[4][0] = F[0];
            Fy[4][1] = F[2];
            Fy[4][2] = F[1];
            Fy[4][3] = F[3];
        }
        // ---- x-faces of output row r ----------------------------------
        if (out_row && tid < Wc + 5) {
            const T *row = ring + RG::slot(r) * (NC * STRIDE) + tid;
            T st[NS][NC];
#pragma unroll
            for (int q = 0; q < NS; ++q)
#pragma unroll
                for (int c = 0; c < NC; ++c) st[q][c] = row[c * STRIDE + q];
            T F[NC];
            ok = face_flux<T, NC, R>(st, tb, F) && ok;
#pragma unroll
            for (int c = 0; c < NC; ++c) Fx[c * NT + tid] = F[c];
        }
        __syncthreads();
        // ---- correction, divergence, stage combination ----------------
        if (s >= s_begin + 4 && col_ok) {
            T fyc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) fyc[c] = corrected<T>(Fy[0][c], Fy[1][c], Fy[2][c], Fy[3][c], Fy[4][c]);
            if (out_row) {
                const T *urow = ring + RG::slot(r) * (NC * STRIDE) + G + tid;
                T res[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T *fx = Fx + c * NT + tid;
                    const T fxp = corrected<T>(fx[1], fx[2], fx[3], fx[4], fx[5]);
                    const T fxm = corrected<T>(fx[0], fx[1], fx[2], fx[3], fx[4]);
                    const T L = -(fxp - fxm) * idx[0] - (fyc[c] - fy_prev[c]) * idx[1];
                    if (a.mode == 0) {
                        res[c] = L;
                    } else {
                        const T v = fma(dt, L, urow[c * STRIDE]);
                        res[c] = a.a0 != T(0) ? fma(a.a0, u0[c], a.b * v) : a.b * v;
                    }
                }
                T *o = a.out + (long)r * nx + x0 + tid;
#pragma unroll
                for (int c = 0; c < NC; ++c) o[c * plane] = res[c];
                if (a.rate) {
                    T rx, ry;
                    rates2d<T>(res, tb.gamma, idx, rx, ry);
                    rmx = Num<T>::fmax(rmx, rx);
                    rmy = Num<T>::fmax(rmy, ry);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) fy_prev[c] = fyc[c];
        }
        cp_async_wait_all();
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void finish_block(const StageArgs<T> &a, T r0, T r1, T r2, bool ok)
{
    if (a.rate) {
        double v0 = (double)r0, v1 = (double)r1, v2 = (double)r2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 = fmax(v0, __shfl_xor_sync(0xffffffffu, v0, o));
            v1 = fmax(v1, __shfl_xor_sync(0xffffffffu, v1, o));
            v2 = fmax(v2, __shfl_xor_sync(0xffffffffu, v2, o));
        }
        if ((threadIdx.x & 31) == 0) {
            // non-negative doubles order like their bit patterns; NaN wins (all ones exponent)
            atomicMax(a.rate + 0, (unsigned long long)__double_as_longlong(v0));
            atomicMax(a.rate + 1, (unsigned long long)__double_as_longlong(v1));
            atomicMax(a.rate + 2, (unsigned long long)__double_as_longlong(v2));
        }
    }
    if (__any_sync(0xffffffffu, !ok) && (threadIdx.x & 31) == 0) atomicOr(a.flags, 1);
}

template <typename T, int R, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) stage2d_kernel(StageArgs<T> a, FaceTables<T, R> tb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const T dt = a.dt_dev ? (T)(*a.dt_dev) : (T)a.dt;
    T rmx = T(0), rmy = T(0);
    bool ok = true;
    // Balanced persistent schedule: the strips' rows, laid end to end
    // (strip-major), are split into gridDim.x equal ranges; a range that
    // crosses a strip boundary becomes two segments.
    const int ny = a.n[1];
    const long long total = (long long)a.nstrips * ny;
    long long u = total * blockIdx.x / gridDim.x;
    const long long uend = total * (blockIdx.x + 1) / gridDim.x;
    while (u < uend) {
        const int strip = (int)(u / ny);
        const int y0 = (int)(u - (long long)strip * ny);
        const int y1 = (int)min((long long)ny, y0 + (uend - u));
        stage2d_segment<T, R, NT>(a, tb, strip, y0, y1, smem, dt, rmx, rmy, ok);
        u += y1 - y0;
    }
    finish_block<T>(a, rmx, rmy, T(0), ok);
}

// ---------------------------------------------------------------------------
// 1D: a CTA owns a segment of W <= NT-5 cells; the segment and its ghost
// cells are staged in shared memory, the W+5 faces evaluated one per thread,
// corrected, differenced and combined.
template <typename T, int R, int NT>
constexpr size_t stage1d_smem_bytes()
{
    return sizeof(T) * (size_t)(3 * (NT - 5 + 2 * (R + 3)) + 3 * NT);
}

template <typename T, int R, int NT>
__global__ void __launch_bounds__(NT) stage1d_kernel(StageArgs<T> a, FaceTables<T, R> tb)
{
    constexpr int G = R + 3, NC = 3, NS = 2 * R + 2;
    constexpr int STRIDE = NT - 5 + 2 * G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *row = reinterpret_cast<T *>(smem_raw);  // [NC][STRIDE]
    T *Fx = row + NC * STRIDE;                 // [NC][NT]
    const T dt = a.dt_dev ? (T)(*a.dt_dev) : (T)a.dt;
    const int tid = threadIdx.x;
    const int nx = a.n[0];
    T rmx = T(0);
    bool ok = true;
    for (int item = blockIdx.x; item < a.nstrips; item += gridDim.x) {
        const int x0 = item * a.W;
        const int Wc = min(a.W, nx - x0);
        for (int col = tid; col < Wc + 2 * G; col += NT) {
            const int gx = bc_map(x0 - G + col, nx, a.per[0]);
#pragma unroll
            for (int c = 0; c < NC; ++c) row[c * STRIDE + col] = a.U[(long)c * nx + gx];
        }
        __syncthreads();
        if (tid < Wc + 5) {
            T st[NS][NC];
#pragma unroll
            for (int q = 0; q < NS; ++q)
#pragma unroll
                for (int c = 0; c < NC; ++c) st[q][c] = row[c * STRIDE + tid + q];
            T F[NC];
            ok = face_flux<T, NC, R>(st, tb, F) && ok;
#pragma unroll
            for (int c = 0; c < NC; ++c) Fx[c * NT + tid] = F[c];
        }
        __syncthreads();
        if (tid < Wc) {
            T res[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T *fx = Fx + c * NT + tid;
                const T L = -(corrected<T>(fx[1], fx[2], fx[3], fx[4], fx[5]) -
                              corrected<T>(fx[0], fx[1], fx[2], fx[3], fx[4])) * a.idx[0];
                if (a.mode == 0) {
                    res[c] = L;
                } else {
                    const T v = fma(dt, L, row[c * STRIDE + G + tid]);
                    res[c] = a.a0 != T(0) ? fma(a.a0, a.U0[(long)c * nx + x0 + tid], a.b * v) : a.b * v;
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) a.out[(long)c * nx + x0 + tid] = res[c];
            if (a.rate) {
                T ir = Num<T>::rcp(res[0]);
                T vx = res[1] * ir;
                T pr = (tb.gamma - T(1)) * (res[2] - T(0.5) * res[1] * vx);
                T cc = Num<T>::sqrt(Num<T>::fmax(tb.gamma * pr * ir, T(0)));
                rmx = Num<T>::fmax(rmx, (Num<T>::fabs(vx) + cc) * a.idx[0]);
            }
        }
        __syncthreads();
    }
    finish_block<T>(a, rmx, T(0), T(0), ok);
}

// Maximum of (|u_d| + c)/dx_d over all cells (for the CFL time step).
template <typename T, int NC>
__global__ void __launch_bounds__(256) max_rate_kernel(const T *U, long ncell, StageArgs<T> a, T gam)
{
    T r[3] = {T(0), T(0), T(0)};
    for (long l = blockIdx.x * (long)blockDim.x + threadIdx.x; l < ncell; l += (long)gridDim.x * blockDim.x) {
        T u[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = U[c * ncell + l];
        T ir = Num<T>::rcp(u[0]);
        T m2 = T(0);
#pragma unroll
        for (int d = 1; d < NC - 1; ++d) m2 = fma(u[d], u[d], m2);
        T pr = (gam - T(1)) * (u[NC - 1] - T(0.5) * m2 * ir);
        T c = Num<T>::sqrt(Num<T>::fmax(gam * pr * ir, T(0)));
#pragma unroll
        for (int d = 0; d < NC - 2; ++d) r[d] = Num<T>::fmax(r[d], (Num<T>::fabs(u[1 + d] * ir) + c) * a.idx[d]);
    }
    finish_block<T>(a, r[0], r[1], r[2], true);
}

// dt = cfl / sum_d rate_d, then the rate accumulators are cleared for the next use.
__global__ void dt_from_rate_kernel(unsigned long long *rate, int ndim, double cfl, double *dt_dev);

}  // namespace gpweno
