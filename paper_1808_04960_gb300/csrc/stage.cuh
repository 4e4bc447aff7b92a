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

// Stage modes.  The SSP-RK3 step is carried in increment form,
//   D_1 = dt L(U^n),  D_2 = 1/4 (D_1 + dt L(U^n + D_1)),  D_3 = 2/3 (D_2 + dt L(U^n + D_2)),
//   U^{n+1} = U^n + D_3,
// which is the Shu-Osher form rewritten with U^(k) = U^n + D_k: increments are
// stored with their own relative precision, and the final sum is compensated
// (TwoSum) with a running remainder `lo`, so state rounding does not
// accumulate over many steps.
enum StageMode { kModeRHS = 0, kModeIncrement = 1, kModeFinal = 2, kModePartial = 3 };
// kModePartial (3D only): the xy-plane kernel writes its part of L, -(div_x/dx + div_y/dy),
// to `out`; the z-marching kernel adds the z part and applies modes 0-2.

template <typename T>
struct StageArgs {
    const T *U;                // stencil state of this stage, SoA [nc][nz][ny][nx]
    const T *U0;               // U^n at the output cell (modes 1, 2); may equal U
    const T *Din;              // previous increment at the output cell (null = 0)
    T *Dout;                   // mode 1: D_k = b (Din + dt L); may equal Din
    T *Vout;                   // mode 1: U^n + D_k (next stage's stencil state)
    T *out;                    // mode 0: L(U); mode 2: U^{n+1} (may equal U0)
    T *lo;                     // mode 2: compensation remainder in/out (null: none)
    int n[3];                  // cells per dimension (x, y, z)
    int per[3];                // periodic flag per dimension
    T idx[3];                  // 1/dx per dimension
    T b;                       // stage weight b_k
    int mode;                  // StageMode
    int u0_is_stencil;         // U0 == U: take U^n from the staged stencil data
    long cstride;              // distance between components (cells of the whole grid)
    const T *P;                // z kernel: x+y part of L written by the plane kernel
    const double *dt_dev;      // device dt (or null: use dt)
    double dt;
    unsigned long long *rate;  // if non-null: atomic max of (|u_d| + c)/dx_d of the result (double bits)
    int *flags;                // bit 0: non-physical state met
    int W, nstrips, H, nseg;   // schedule: strip width, #strips, segment height, #segments
    // Slab decomposition: along the slowest dimension (slab_dim = ndim-1, or -1 if no side is
    // external) the ghost layers of an external side come from a caller-filled halo buffer of
    // G = R+3 layers, [nc][G][layer], layer k = the k-th cell beyond the side in increasing order.
    int slab_dim;
    int ext[2];                // low / high side external
    const T *halo[2];          // halo buffers of the low / high side
};

// Source of layer g (a cell index along the slab dimension, possibly a ghost) of a
// state whose layers are `unit` cells apart: the state itself, or an external halo.
// `cs` receives the distance between components at that source.
template <typename T>
__device__ __forceinline__ const T *layer_src(const StageArgs<T> &a, const T *U, int g, int n, int per, long unit,
                                              int G, long &cs)
{
    if (g < 0 && a.ext[0]) {
        cs = (long)G * unit;
        return a.halo[0] + (long)(g + G) * unit;
    }
    if (g >= n && a.ext[1]) {
        cs = (long)G * unit;
        return a.halo[1] + (long)(g - n) * unit;
    }
    cs = a.cstride;
    return U + (long)bc_map(g, n, per) * unit;
}

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

// Bounds-checked build (-DGPWENO_CHECKED; the tests build it as a library of its own): every
// shared-memory and global access of the stage kernels is first checked against the extent of
// its array; a violation sets bit `site` of the plan's flag word and skips the access (a read
// yields zero).  The default build compiles the checks away.
#ifdef GPWENO_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
enum CheckSite {
    kChkRingWrite = 1,   // staging copy into the shared ring (2D, xy-planes)
    kChkStateRead = 2,   // global source of a staging copy (stage state or halo buffer)
    kChkRingRead = 3,    // stencil or U^n read from the ring
    kChkFaceWrite = 4,   // staged x-face fluxes
    kChkFaceRead = 5,
    kChkEpiRead = 6,     // U^n, increment, remainder or partial L of an output cell
    kChkEpiWrite = 7,    // stage outputs
    kChkZRing = 8,       // z kernel: shared ring
    kChkZState = 9,      // z kernel: staging source
    kChkLine = 10,       // 1D kernel: shared row and face arrays
    kChkLineState = 11   // 1D kernel: staging source
};

__device__ __forceinline__ bool chk(long long i, long long n, int site, int *flags)
{
    if constexpr (kChecked) {
        if (i < 0 || i >= n) {
            atomicOr(flags, 1 << site);
            return false;
        }
    }
    return true;
}

// Checked build: does p point into the stage state (ext_state elements) or into a registered
// halo buffer (ext_halo elements each)?
template <typename T>
__device__ __forceinline__ bool src_ok(const StageArgs<T> &a, const T *p, long ext_state, long ext_halo, int site)
{
    if constexpr (kChecked) {
        const bool in = (p >= a.U && p < a.U + ext_state) ||
                        (a.halo[0] != nullptr && p >= a.halo[0] && p < a.halo[0] + ext_halo) ||
                        (a.halo[1] != nullptr && p >= a.halo[1] && p < a.halo[1] + ext_halo);
        if (!in) atomicOr(a.flags, 1 << site);
        return in;
    }
    return true;
}

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

template <typename T, int R, int NT, int NC = 4>
constexpr size_t stage2d_smem_bytes()
{
    using RG = Ring2D<R, NT>;
    return sizeof(T) * (size_t)(RG::ROWS * NC * RG::STRIDE + 2 * NC * NT);
}

// Error-free sum a + b = s + e (Knuth's TwoSum).
template <typename T>
__device__ __forceinline__ T two_sum(T a, T b, T &e)
{
    const T s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// Epilogue of one cell and component: L is the RHS, u the stencil-state value of
// the cell, u0/din/lo the prefetched U^n, previous increment and remainder.
// Returns the value whose wavespeed the CFL reduction sees (mode 2: U^{n+1}).
template <typename T>
__device__ __forceinline__ T stage_epilogue(const StageArgs<T> &a, long cell, T L, T u0, T din, T lo, T dt,
                                            long extent)
{
    if (!chk(cell, extent, kChkEpiWrite, a.flags)) return L;
    if (a.mode == kModeRHS) {
        a.out[cell] = L;
        return L;
    }
    const T inc = a.b * fma(dt, L, din);
    if (a.mode == kModeIncrement) {
        a.Dout[cell] = inc;
        a.Vout[cell] = u0 + inc;
        return u0 + inc;
    }
    if (a.lo) {
        T e;
        const T t = inc + lo;
        const T snew = two_sum<T>(u0, t, e);
        a.out[cell] = snew;
        a.lo[cell] = e;
        return snew;
    }
    const T snew = u0 + inc;
    a.out[cell] = snew;
    return snew;
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

// One segment: rows [y0, y1) of strip `strip` of the xy-plane starting at cell offset zoff.
// NC = 4 (2D) or 5 (an xy-plane of a 3D grid).
// ONE_SITE: evaluate the y- and x-face through one copy of the face routine (a
// loop of two passes) instead of two inlined copies.  Two copies let the compiler
// interleave the two independent faces (faster for the 2D kernels, the FP32 batch
// included); one copy halves the code, which pays in the FP64 batch (fewer spills
// with three radii in one kernel) and in 3D.
template <typename T, int R, int NT, int NC = 4, int VAR = 0, bool ONE_SITE = false>
__device__ __forceinline__ void stage2d_segment(const StageArgs<T> &a, const FaceTables<T, R> &tb, int strip, int y0,
                                                int y1, T *smem, T dt, T &rmx, T &rmy, bool &ok, long zoff = 0)
{
    using RG = Ring2D<R, NT>;
    constexpr int G = RG::G, ROWS = RG::ROWS, STRIDE = RG::STRIDE;
    constexpr int NS = 2 * R + 2;
    // FP32 2D kernel: the four components of a ring element and of a staged face flux sit side
    // by side (one 16-byte shared load per stencil cell or face flux); otherwise one array per
    // component.  The one-site loop (3D planes, FP64 batches), the FD-Flux form and GP-AO keep the
    // per-component arrays: there the aligned register quads of 16-byte loads cost spills.
    constexpr bool VEC = std::is_same<T, float>::value && NC == 4 && !ONE_SITE && (VAR & (kVarFdFlux | kVarAo)) == 0;
    T *ring = smem;                              // [ROWS][NC][STRIDE], or [ROWS][STRIDE][4] (VEC)
    T *FA = smem + ROWS * NC * STRIDE;           // [NC][NT] (or [NT][4]): x-face A = F_{s+1/2} - F(U_s)
    T *FB = FA + NC * NT;                        // [NC][NT] (or [NT][4]): x-face B = F(U_{s+1}) - F(U_s)
    // offset of component c of element col in the ring row starting at `base`, and of a face flux
    auto ro = [](int base, int col, int c) { return VEC ? base + col * 4 + c : base + c * STRIDE + col; };
    auto fo = [](int t, int c) { return VEC ? t * 4 + c : c * NT + t; };
    // the NC values of element col of a ring row (VEC: one 16-byte load)
    auto ring_elem = [&](int base, int col, T (&v)[NC]) {
        if constexpr (kChecked) {
            const int first = VEC ? base + col * 4 : base + col, last = VEC ? first + 3 : first + (NC - 1) * STRIDE;
            if (!chk(first, ROWS * NC * STRIDE, kChkRingRead, a.flags) ||
                !chk(last, ROWS * NC * STRIDE, kChkRingRead, a.flags)) {
#pragma unroll
                for (int c = 0; c < NC; ++c) v[c] = T(0);
                return;
            }
        }
        if constexpr (VEC) {
            const float4 q = *reinterpret_cast<const float4 *>(ring + base + col * 4);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] = ring[base + c * STRIDE + col];
        }
    };
    // one ring element (checked build: in bounds or zero)
    auto ring_at = [&](int i) -> T { return chk(i, ROWS * NC * STRIDE, kChkRingRead, a.flags) ? ring[i] : T(0); };
    auto stage_face = [&](T *F, int t, const T (&v)[NC]) {
        if (!chk(t, NT, kChkFaceWrite, a.flags)) return;
        if constexpr (VEC) {
            *reinterpret_cast<float4 *>(F + t * 4) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c * NT + t] = v[c];
        }
    };
    const int tid = threadIdx.x;
    const int nx = a.n[0], ny = a.n[1];
    const long plane = a.cstride;
    const int x0 = strip * a.W;
    const int Wc = min(a.W, nx - x0);
    const int s_begin = y0 - 3, s_end = y1 + 1;
    const int rowlen = Wc + 2 * G;
    const T idx[3] = {a.idx[0], a.idx[1], a.idx[2]};

    // one staging copy (checked build: destination in the ring, source in the state or a halo)
    auto stage_copy = [&](T *dst, const T *src) {
        if (!chk(dst - ring, ROWS * NC * STRIDE, kChkRingWrite, a.flags) ||
            !src_ok<T>(a, src, (long)NC * plane, (long)NC * G * nx, kChkStateRead))
            return;
        cp_async_elem(dst, src);
    };
    auto load_row = [&](int g) {
        T *dst = ring + RG::slot(g) * (NC * STRIDE);
        if ((VAR & kVarSlab) != 0 && NC == 4 && a.slab_dim == 1 && ((g < 0 && a.ext[0]) || (g >= ny && a.ext[1]))) {
            // a ghost row of an external side: from the halo buffer [nc][G][nx]
            const T *src = g < 0 ? a.halo[0] + (long)(g + G) * nx : a.halo[1] + (long)(g - ny) * nx;
            for (int col = tid; col < rowlen; col += NT) {
                const int gx = bc_map(x0 - G + col, nx, a.per[0]);
#pragma unroll
                for (int c = 0; c < NC; ++c) stage_copy(dst + ro(0, col, c), src + (long)c * G * nx + gx);
            }
            return;
        }
        const int gy = bc_map(g, ny, a.per[1]);
        const T *src = a.U + zoff + (long)gy * nx;
        for (int col = tid; col < rowlen; col += NT) {
            const int gx = bc_map(x0 - G + col, nx, a.per[0]);
#pragma unroll
            for (int c = 0; c < NC; ++c) stage_copy(dst + ro(0, col, c), src + c * plane + gx);
        }
    };

    // prologue: rows needed by the first y-face
    for (int g = s_begin - R; g <= s_begin + 1 + R; ++g) load_row(g);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    // per column: flux jumps dF_{s'} = F_{s'+1/2} - F_{s'-1/2} across the last five rows,
    // and A, B of the previous y-face
    T Dy[5][NC], Ap[NC], Bp[NC];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) Dy[k][c] = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) Ap[c] = Bp[c] = T(0);

    for (int s = s_begin; s <= s_end; ++s) {
        if (s < s_end) load_row(s + 2 + R);
        cp_async_commit();
        const int r = s - 2;
        const bool out_row = r >= y0;
        const bool col_ok = tid < Wc;

        // U^n, previous increment and remainder of this thread's output cell,
        // in flight during the face work
        T u0[NC], din[NC], lov[NC];
        const long cell = zoff + (long)r * nx + x0 + tid;
        const bool epi = out_row && col_ok && (a.mode == kModeIncrement || a.mode == kModeFinal);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool in = !epi || chk(c * plane + cell, (long)NC * plane, kChkEpiRead, a.flags);
            u0[c] = (epi && in && !a.u0_is_stencil) ? a.U0[c * plane + cell] : T(0);
            din[c] = (epi && in && a.Din) ? a.Din[c * plane + cell] : T(0);
            lov[c] = (epi && in && a.lo && a.mode == kModeFinal) ? a.lo[c * plane + cell] : T(0);
        }

        if constexpr (ONE_SITE) {
            // ---- y-face s+1/2 of column tid (pass 0) and x-face tid of output row r (pass 1),
            // through one copy of the face routine ------------------------------
            const bool do_y = col_ok, do_x = out_row && tid < Wc + 5;
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 0 ? !do_y : !do_x) continue;
                // stencil element (q, c): ring + off[q] + comp[c] * STRIDE, normal-first
                static_assert(!VEC, "the one-site loop keeps one array per component");
                int off[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    off[q] = pass == 0 ? RG::slot(s - R + q) * (NC * STRIDE) + G + tid : RG::slot(r) * (NC * STRIDE) + tid + q;
                T st[NS][NC];
#pragma unroll
                for (int q = 0; q < NS; ++q)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        // a y-face's normal is the second velocity: (rho, rho v, rho u, [rho w], E)
                        const int cc = pass == 0 ? (c == 1 ? 2 : (c == 2 ? 1 : c)) : c;
                        st[q][c] = ring_at(off[q] + cc * STRIDE);
                    }
                T An[NC], Bn[NC];
                ok = face_eval<T, NC, R, VAR>(st, tb, An, Bn) && ok;
                if (pass == 0) {
                    T Ac[NC], Bc[NC];   // back to natural order
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int pc = c == 1 ? 2 : (c == 2 ? 1 : c);
                        Ac[c] = An[pc];
                        Bc[c] = Bn[pc];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int c = 0; c < NC; ++c) Dy[k][c] = Dy[k + 1][c];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        Dy[4][c] = Ac[c] - Ap[c] + Bp[c];   // jump across row s (valid once s > s_begin)
                        Ap[c] = Ac[c];
                        Bp[c] = Bc[c];
                    }
                } else {
                    stage_face(FA, tid, An);
                    stage_face(FB, tid, Bn);
                }
            }
        } else {
            // ---- y-face s+1/2 of column tid --------------------------------
            if (col_ok) {
                T st[NS][NC];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int base = RG::slot(s - R + q) * (NC * STRIDE);
                    // normal-first for a y-face: (rho, rho v, rho u, [rho w], E)
                    if constexpr (VEC) {
                        T v[NC];
                        ring_elem(base, G + tid, v);
#pragma unroll
                        for (int c = 0; c < NC; ++c) st[q][c] = v[c == 1 ? 2 : (c == 2 ? 1 : c)];
                    } else {
#pragma unroll
                        for (int c = 0; c < NC; ++c) st[q][c] = ring_at(ro(base, G + tid, c == 1 ? 2 : (c == 2 ? 1 : c)));
                    }
                }
                T An[NC], Bn[NC];
                ok = face_eval<T, NC, R, VAR>(st, tb, An, Bn) && ok;
                T Ac[NC], Bc[NC];   // back to natural order
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int pc = c == 1 ? 2 : (c == 2 ? 1 : c);
                    Ac[c] = An[pc];
                    Bc[c] = Bn[pc];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) Dy[k][c] = Dy[k + 1][c];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    Dy[4][c] = Ac[c] - Ap[c] + Bp[c];   // jump across row s (valid once s > s_begin)
                    Ap[c] = Ac[c];
                    Bp[c] = Bc[c];
                }
            }
            // ---- x-faces of output row r ----------------------------------
            if (out_row && tid < Wc + 5) {
                const int base = RG::slot(r) * (NC * STRIDE);
                T st[NS][NC];
#pragma unroll
                for (int q = 0; q < NS; ++q) ring_elem(base, tid + q, st[q]);
                T An[NC], Bn[NC];
                ok = face_eval<T, NC, R, VAR>(st, tb, An, Bn) && ok;
                stage_face(FA, tid, An);
                stage_face(FB, tid, Bn);
            }
        }
        __syncthreads();
        // ---- divergence and stage combination -------------------------
        if (out_row && col_ok && chk(tid + 5, NT, kChkFaceRead, a.flags)) {
            const int ubase = RG::slot(r) * (NC * STRIDE);
            T un4[NC];
            if constexpr (VEC) {
                if (a.u0_is_stencil) ring_elem(ubase, G + tid, un4);
            }
            // x-faces t = tid..tid+5 are s' = x-3..x+2 around cell x = x0 + tid; the flux jumps
            // dF_k = A_{k+1} - A_k + B_k across the five cells around x (VEC: all components
            // from 16-byte loads, rolling over k; otherwise one component at a time)
            T dxk[VEC ? 5 : 1][NC];
            if constexpr (VEC) {
                float4 q = *reinterpret_cast<const float4 *>(FA + tid * 4);
                T prev[NC] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    q = *reinterpret_cast<const float4 *>(FA + (tid + k + 1) * 4);
                    const float4 w = *reinterpret_cast<const float4 *>(FB + (tid + k) * 4);
                    const T cur[NC] = {q.x, q.y, q.z, q.w}, b[NC] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        dxk[k][c] = cur[c] - prev[c] + b[c];
                        prev[c] = cur[c];
                    }
                }
            }
            T res[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T dx[5];
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    dx[k] = VEC ? dxk[VEC ? k : 0][c]
                                : FA[fo(tid + k + 1, c)] - FA[fo(tid + k, c)] + FB[fo(tid + k, c)];
                const T divx = flux_divergence<T, VAR>(dx[0], dx[1], dx[2], dx[3], dx[4]);
                const T divy = flux_divergence<T, VAR>(Dy[0][c], Dy[1][c], Dy[2][c], Dy[3][c], Dy[4][c]);
                const T L = -fma(divx, idx[0], divy * idx[1]);
                if (NC == 5 || a.mode == kModePartial) {
                    if (chk(c * plane + cell, (long)NC * plane, kChkEpiWrite, a.flags)) a.out[c * plane + cell] = L;
                    res[c] = L;
                } else {
                    const T un = a.u0_is_stencil ? (VEC ? un4[c] : ring_at(ro(ubase, G + tid, c))) : u0[c];
                    res[c] = stage_epilogue<T>(a, c * plane + cell, L, un, din[c], lov[c], dt, (long)NC * plane);
                }
            }
            if (NC == 4 && a.rate && a.mode == kModeFinal) {
                T rx, ry;
                rates2d<T>(reinterpret_cast<const T(&)[4]>(res), tb.gamma, idx, rx, ry);
                rmx = Num<T>::fmax(rmx, rx);
                rmy = Num<T>::fmax(rmy, ry);
            }
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

// Programmatic dependent launch: wait until the stream's preceding grid has
// finished and its writes are visible (a no-op without a programmatic
// dependency), then allow the stream's next kernel to be scheduled, so that its
// launch overlaps this grid's tail.  Every global access comes after this.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// First row of CTA b in the cost-balanced split of the strip-major row order
// [0, total) over `grid` CTAs.  A row costs 2 (one x- and one y-face per
// column) and every strip start inside a range costs 5 more (the warm-up
// y-face rows of a new segment), so rows [0, u) cost 2u + 5 floor((u-1)/ny);
// CTA b starts at the first row where that reaches b/grid of the total.
// Non-decreasing in b, 0 at b = 0 and total at b = grid, so the ranges
// [start(b), start(b+1)) partition the rows.
__device__ __forceinline__ long long balanced_start(int b, int grid, long long total, int ny, int nstrips)
{
    if (b <= 0) return 0;
    if (b >= grid) return total;
    const long long ctot = 2 * total + 5 * ((total - 1) / ny);
    const long long c = (ctot * b + grid / 2) / grid;
    for (int k = 0; k < nstrips; ++k) {
        const long long lo = (long long)k * ny, hi = lo + ny;
        if (2 * hi + 5LL * k >= c) return min(max((c - 5LL * k + 1) / 2, lo), hi);
    }
    return total;
}

// MINB: resident CTAs per SM the register budget is cut for (the default four 128-thread CTAs
// in FP32 at 128 registers; three give the compiler ~150 registers, which pays on small grids,
// see the host's choice in launch_stage_R).
template <typename T, int R, int NT, int VAR = 0, int MINB = (sizeof(T) == 4 ? 512 : 256) / NT>
__global__ void __launch_bounds__(NT, MINB) stage2d_kernel(StageArgs<T> a, TablesFor<T, R, VAR> tb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    pdl_enter();
    const T dt = a.dt_dev ? (T)(*a.dt_dev) : (T)a.dt;
    T rmx = T(0), rmy = T(0);
    bool ok = true;
    // Persistent schedule: the strips' rows, laid end to end (strip-major),
    // are split into gridDim.x ranges of equal estimated cost; a range that
    // crosses a strip boundary becomes two segments.
    const int ny = a.n[1];
    const long long total = (long long)a.nstrips * ny;
    long long u = balanced_start(blockIdx.x, gridDim.x, total, ny, a.nstrips);
    const long long uend = balanced_start(blockIdx.x + 1, gridDim.x, total, ny, a.nstrips);
    while (u < uend) {
        const int strip = (int)(u / ny);
        const int y0 = (int)(u - (long long)strip * ny);
        const int y1 = (int)min((long long)ny, y0 + (uend - u));
        stage2d_segment<T, R, NT, 4, VAR>(a, tb, strip, y0, y1, smem, dt, rmx, rmy, ok);
        u += y1 - y0;
    }
    finish_block<T>(a, rmx, rmy, T(0), ok);
}

// ---------------------------------------------------------------------------
// 3D.  Each stage is two launches: the xy-plane kernel below runs the 2D
// column-strip marching routine (5 components) on every z-plane and writes
// -(div_x/dx + div_y/dy) to a stage buffer P; the z-marching kernel then walks
// contiguous runs of xy-columns along z, evaluates each z-face once, adds
// -div_z/dz to P and applies the stage update.  P is a buffer the update later
// overwrites cell by cell (each cell reads its own P first), so 3D needs no
// scratch beyond 2D's.
template <typename T, int R, int NT, int VAR = 0>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 512 : 256) / NT) plane3d_kernel(StageArgs<T> a, TablesFor<T, R, VAR> tb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    pdl_enter();
    T rmx = T(0), rmy = T(0);
    bool ok = true;
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long per_plane = (long)a.nstrips * ny;
    const long total = per_plane * nz;
    long long u = (long long)total * blockIdx.x / gridDim.x;
    const long long uend = (long long)total * (blockIdx.x + 1) / gridDim.x;
    while (u < uend) {
        const int z = (int)(u / per_plane);
        const long rem = u - (long long)z * per_plane;
        const int strip = (int)(rem / ny);
        const int y0 = (int)(rem - (long)strip * ny);
        const int y1 = (int)min((long long)ny, y0 + (uend - u));
        stage2d_segment<T, R, NT, 5, VAR, true>(a, tb, strip, y0, y1, smem, T(0), rmx, rmy, ok, (long)z * nx * ny);
        u += y1 - y0;
    }
    if (__any_sync(0xffffffffu, !ok) && (threadIdx.x & 31) == 0) atomicOr(a.flags, 1);
}

template <int R>
struct RingZ {
    static constexpr int LOW = R > 2 ? R : 2;
    static constexpr int NEEDED = LOW + R + 3;
    static constexpr int ROWS = NEEDED <= 8 ? 8 : 16;
    static __device__ __forceinline__ int slot(int g) { return g & (ROWS - 1); }
};

template <typename T, int R, int NT>
constexpr size_t stagez_smem_bytes()
{
    return sizeof(T) * (size_t)(RingZ<R>::ROWS * 5 * NT);
}

template <typename T>
__device__ __forceinline__ void rates3d(const T (&u)[5], T gam, const T (&idx)[3], T &rx, T &ry, T &rz)
{
    const T ir = Num<T>::rcp(u[0]);
    const T vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
    const T pr = (gam - T(1)) * (u[4] - T(0.5) * (u[1] * vx + u[2] * vy + u[3] * vz));
    const T c = Num<T>::sqrt(Num<T>::fmax(gam * pr * ir, T(0)));
    rx = (Num<T>::fabs(vx) + c) * idx[0];
    ry = (Num<T>::fabs(vy) + c) * idx[1];
    rz = (Num<T>::fabs(vz) + c) * idx[2];
}

// z-marching over columns [c0, c0+NT) of the flattened xy-plane, planes [z0, z1).
template <typename T, int R, int NT, int VAR = 0>
__device__ __forceinline__ void stagez_segment(const StageArgs<T> &a, const FaceTables<T, R> &tb, long c0, int z0,
                                               int z1, T *ring, T dt, T (&rm)[3], bool &ok)
{
    using RZ = RingZ<R>;
    constexpr int NC = 5, NS = 2 * R + 2;
    const int tid = threadIdx.x;
    const int nz = a.n[2];
    const long plane = (long)a.n[0] * a.n[1];
    const long cs = a.cstride;
    const long col = c0 + tid;
    const bool col_ok = col < plane;
    const int s_begin = z0 - 3, s_end = z1 + 1;
    const T idx[3] = {a.idx[0], a.idx[1], a.idx[2]};

    auto load_plane = [&](int g) {
        if (!col_ok) return;
        constexpr int G = R + 3;
        T *dst = ring + RZ::slot(g) * (NC * NT) + tid;
        long ccs = cs;
        const T *src = ((VAR & kVarSlab) != 0 && a.slab_dim == 2 ? layer_src<T>(a, a.U, g, nz, a.per[2], plane, G, ccs)
                                                                 : a.U + (long)bc_map(g, nz, a.per[2]) * plane) +
                       col;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (chk(dst + c * NT - ring, RZ::ROWS * NC * NT, kChkZRing, a.flags) &&
                src_ok<T>(a, src + c * ccs, NC * cs, (long)NC * G * plane, kChkZState))
                cp_async_elem(dst + c * NT, src + c * ccs);
    };
    for (int g = s_begin - R; g <= s_begin + 1 + R; ++g) load_plane(g);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    T Dz[5][NC], Ap[NC], Bp[NC];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) Dz[k][c] = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) Ap[c] = Bp[c] = T(0);

    for (int s = s_begin; s <= s_end; ++s) {
        if (s < s_end) load_plane(s + 2 + R);
        cp_async_commit();
        const int r = s - 2;
        const bool out = r >= z0 && col_ok;
        const long cell = (long)r * plane + col;
        T pv[NC], u0[NC], din[NC], lov[NC];
        const bool epi = out && (a.mode == kModeIncrement || a.mode == kModeFinal);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool in = !out || chk(c * cs + cell, NC * cs, kChkEpiRead, a.flags);
            pv[c] = (out && in) ? a.P[c * cs + cell] : T(0);
            u0[c] = (epi && in && !a.u0_is_stencil) ? a.U0[c * cs + cell] : T(0);
            din[c] = (epi && in && a.Din) ? a.Din[c * cs + cell] : T(0);
            lov[c] = (epi && in && a.lo && a.mode == kModeFinal) ? a.lo[c * cs + cell] : T(0);
        }
        if (col_ok) {
            // normal-first for a z-face: (rho, rho w, rho u, rho v, E)
            T st[NS][NC];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const T *rowp = ring + RZ::slot(s - R + q) * (NC * NT) + tid;
                if (!chk(rowp + 4 * NT - ring, RZ::ROWS * NC * NT, kChkZRing, a.flags)) rowp = ring;
                st[q][0] = rowp[0];
                st[q][1] = rowp[3 * NT];
                st[q][2] = rowp[1 * NT];
                st[q][3] = rowp[2 * NT];
                st[q][4] = rowp[4 * NT];
            }
            T An[NC], Bn[NC];
            ok = face_eval<T, NC, R, VAR>(st, tb, An, Bn) && ok;
            const T Ac[NC] = {An[0], An[2], An[3], An[1], An[4]};
            const T Bc[NC] = {Bn[0], Bn[2], Bn[3], Bn[1], Bn[4]};
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) Dz[k][c] = Dz[k + 1][c];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                Dz[4][c] = Ac[c] - Ap[c] + Bp[c];
                Ap[c] = Ac[c];
                Bp[c] = Bc[c];
            }
        }
        if (out) {
            const T *urow = ring + RZ::slot(r) * (NC * NT) + tid;
            if (!chk(urow + 4 * NT - ring, RZ::ROWS * NC * NT, kChkZRing, a.flags)) urow = ring;
            T res[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T divz = flux_divergence<T, VAR>(Dz[0][c], Dz[1][c], Dz[2][c], Dz[3][c], Dz[4][c]);
                const T L = fma(-divz, idx[2], pv[c]);
                const T un = a.u0_is_stencil ? urow[c * NT] : u0[c];
                res[c] = stage_epilogue<T>(a, c * cs + cell, L, un, din[c], lov[c], dt, NC * cs);
            }
            if (a.rate && a.mode == kModeFinal) {
                T rx, ry, rz;
                rates3d<T>(res, tb.gamma, idx, rx, ry, rz);
                rm[0] = Num<T>::fmax(rm[0], rx);
                rm[1] = Num<T>::fmax(rm[1], ry);
                rm[2] = Num<T>::fmax(rm[2], rz);
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
}

template <typename T, int R, int NT, int VAR = 0>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) stagez_kernel(StageArgs<T> a, TablesFor<T, R, VAR> tb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    pdl_enter();
    const T dt = a.dt_dev ? (T)(*a.dt_dev) : (T)a.dt;
    T rm[3] = {T(0), T(0), T(0)};
    bool ok = true;
    const int nz = a.n[2];
    const long plane = (long)a.n[0] * a.n[1];
    const long groups = (plane + NT - 1) / NT;
    const long long total = (long long)groups * nz;
    long long u = total * blockIdx.x / gridDim.x;
    const long long uend = total * (blockIdx.x + 1) / gridDim.x;
    while (u < uend) {
        const long g = (long)(u / nz);
        const int z0 = (int)(u - (long long)g * nz);
        const int z1 = (int)min((long long)nz, z0 + (uend - u));
        stagez_segment<T, R, NT, VAR>(a, tb, g * NT, z0, z1, ring, dt, rm, ok);
        u += z1 - z0;
    }
    finish_block<T>(a, rm[0], rm[1], rm[2], ok);
}

// ---------------------------------------------------------------------------
// 1D: a CTA owns a segment of W <= NT-5 cells; the segment and its ghost
// cells are staged in shared memory, the W+5 faces evaluated one per thread,
// corrected, differenced and combined.
template <typename T, int R, int NT>
constexpr size_t stage1d_smem_bytes()
{
    return sizeof(T) * (size_t)(3 * (NT - 5 + 2 * (R + 3)) + 2 * 3 * NT);
}

template <typename T, int R, int NT, int VAR = 0>
__global__ void __launch_bounds__(NT) stage1d_kernel(StageArgs<T> a, TablesFor<T, R, VAR> tb)
{
    constexpr int G = R + 3, NC = 3, NS = 2 * R + 2;
    constexpr int STRIDE = NT - 5 + 2 * G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *row = reinterpret_cast<T *>(smem_raw);  // [NC][STRIDE]
    T *FA = row + NC * STRIDE;                 // [NC][NT]
    T *FB = FA + NC * NT;                      // [NC][NT]
    pdl_enter();
    const T dt = a.dt_dev ? (T)(*a.dt_dev) : (T)a.dt;
    const int tid = threadIdx.x;
    const int nx = a.n[0];
    T rmx = T(0);
    bool ok = true;
    for (int item = blockIdx.x; item < a.nstrips; item += gridDim.x) {
        const int x0 = item * a.W;
        const int Wc = min(a.W, nx - x0);
        for (int col = tid; col < Wc + 2 * G; col += NT) {
            long cs = nx;
            const T *src = (VAR & kVarSlab) != 0 && a.slab_dim == 0
                               ? layer_src<T>(a, a.U, x0 - G + col, nx, a.per[0], 1, G, cs)
                               : a.U + bc_map(x0 - G + col, nx, a.per[0]);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (chk(col, STRIDE, kChkLine, a.flags) &&
                    src_ok<T>(a, src + c * cs, (long)NC * nx, (long)NC * G, kChkLineState))
                    row[c * STRIDE + col] = src[c * cs];
        }
        __syncthreads();
        if (tid < Wc + 5 && chk(tid + NS - 1, STRIDE, kChkLine, a.flags) && chk(tid, NT, kChkLine, a.flags)) {
            T st[NS][NC];
#pragma unroll
            for (int q = 0; q < NS; ++q)
#pragma unroll
                for (int c = 0; c < NC; ++c) st[q][c] = row[c * STRIDE + tid + q];
            T An[NC], Bn[NC];
            ok = face_eval<T, NC, R, VAR>(st, tb, An, Bn) && ok;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                FA[c * NT + tid] = An[c];
                FB[c * NT + tid] = Bn[c];
            }
        }
        __syncthreads();
        if (tid < Wc && chk(tid + 5, NT, kChkLine, a.flags) && chk(G + tid, STRIDE, kChkLine, a.flags)) {
            T res[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T *fa = FA + c * NT + tid;
                const T *fb = FB + c * NT + tid;
                T dx[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) dx[k] = fa[k + 1] - fa[k] + fb[k];
                const T L = -flux_divergence<T, VAR>(dx[0], dx[1], dx[2], dx[3], dx[4]) * a.idx[0];
                const long cell = (long)c * nx + x0 + tid;
                const bool epi = a.mode != kModeRHS && chk(cell, (long)NC * nx, kChkEpiRead, a.flags);
                const T u0 = a.u0_is_stencil ? row[c * STRIDE + G + tid] : (epi ? a.U0[cell] : T(0));
                const T din = (epi && a.Din) ? a.Din[cell] : T(0);
                const T lov = (epi && a.lo && a.mode == kModeFinal) ? a.lo[cell] : T(0);
                res[c] = stage_epilogue<T>(a, cell, L, u0, din, lov, dt, (long)NC * nx);
            }
            if (a.rate && a.mode == kModeFinal) {
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
