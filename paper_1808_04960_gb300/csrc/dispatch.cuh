// Host-side launch of the stage kernels for one arithmetic type: table
// conversion, schedule (strip width, segment height, grid), kernel selection.
#pragma once
#include <algorithm>

#include "plan.h"
#include "stage.cuh"

namespace gpweno {

// Block size of the 3D z-marching kernel (contiguous runs of 256 xy-columns).
constexpr int kNTz = 256;
// Block size of the xy-sweeping kernels (2D stage, 3D plane).  FP32: 128 threads
// and four CTAs per SM, with the same 128 registers per thread as two 256-thread
// CTAs.  A strip is then at most 123 columns, so every warp of a CTA evaluates
// faces and each of the four SM sub-partitions holds four busy warps.  With 256
// threads and strips narrower than 251 columns (205 at nx = 1024) the eighth warp
// of each CTA idles.  Its sub-partition then carries half the load of the others,
// and a row takes as long as the busiest sub-partition needs.  Measured on GB300:
// +8 % at 1024^2, +6 % at 2048^2, +1 % at 4096^2.  FP64 (255 registers, one
// 256-thread CTA per SM) keeps 256: 128 threads measured 4 % slower.
template <typename T>
constexpr int kNTxy = sizeof(T) == 4 ? 128 : 256;
constexpr int kNT1D = 128;

template <typename T, int R>
FaceTables<T, R> make_tables(const gpweno_plan_s *p)
{
    FaceTables<T, R> t;
    const int S = R + 1;
    for (int m = 0; m < S; ++m)
        for (int j = 0; j < S; ++j) {
            t.wl[m][j] = (T)p->tab.wl[m * S + j];
            t.wr[m][j] = (T)p->tab.wr[m * S + j];
            t.gwl[m][j] = (T)p->tab.gwl[m * S + j];
            t.gwr[m][j] = (T)p->tab.gwr[m * S + j];
        }
    for (int k = 0; k < S; ++k)
        for (int j = 0; j < (R + 2) / 2; ++j) t.Ph[k][j] = (T)p->tab.Ph[k * S + j];
    for (int m = 0; m < S; ++m) {
        t.gl[m] = (T)p->tab.gl[m];
        t.gr[m] = (T)p->tab.gr[m];
        t.sl1[m] = (T)p->tab.sl1[m];
        t.sr1[m] = (T)p->tab.sr1[m];
        t.gsl1[m] = (T)p->tab.gsl1[m];
        t.gsr1[m] = (T)p->tab.gsr1[m];
        t.Psum[m] = (T)p->tab.Psum[m];
    }
    t.eps = (T)p->opts.eps;
    t.gamma = (T)p->gamma;
    t.p = p->opts.p;
    t.flux = p->opts.flux_form;
    return t;
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the stream's preceding kernel finishes; the stage kernels wait for it
// (pdl_enter) before any global access.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Tables of a scheme variant: GP-AO adds its own on top of the GP-WENO ones.
template <typename T, int R, int VAR>
TablesFor<T, R, VAR> make_tables_var(const gpweno_plan_s *p)
{
    if constexpr ((VAR & kVarAo) != 0) {
        using AT = AoFaceTables<T, R>;
        constexpr int NH = AT::NH, NL = AT::NL;
        AT t;
        std::memset(&t, 0, sizeof(t));
        static_cast<FaceTables<T, R> &>(t) = make_tables<T, R>(p);
        const AoTables &a = p->ao;
        for (int j = 0; j < NH; ++j) {
            t.whl[j] = (T)a.w_hi_l[j];
            t.whr[j] = (T)a.w_hi_r[j];
        }
        t.shl = (T)a.s_hi_l;
        t.shr = (T)a.s_hi_r;
        if (R == 3) {
            for (int j = 0; j < NL; ++j) {
                t.wll[j] = (T)a.w_lo_l[j];
                t.wlr[j] = (T)a.w_lo_r[j];
            }
            t.sll = (T)a.s_lo_l;
            t.slr = (T)a.s_lo_r;
            for (int k = 0; k < NL; ++k) {
                for (int j = 0; j < (NL + 1) / 2; ++j) t.Plo[k][j] = (T)a.Ph_lo[k * NL + j];
                t.Psum_lo[k] = (T)a.Psum_lo[k];
            }
        }
        for (int m = 0; m < 3; ++m) {
            for (int j = 0; j < 3; ++j) {
                t.w3l[m][j] = (T)a.w3_l[3 * m + j];
                t.w3r[m][j] = (T)a.w3_r[3 * m + j];
            }
            t.s3l[m] = (T)a.s3_l[m];
            t.s3r[m] = (T)a.s3_r[m];
        }
        for (int k = 0; k < NH; ++k) {
            for (int j = 0; j < (NH + 1) / 2; ++j) t.Phi[k][j] = (T)a.Ph_hi[k * NH + j];
            t.Psum_hi[k] = (T)a.Psum_hi[k];
        }
        for (int k = 0; k < 3; ++k) {
            for (int j = 0; j < 2; ++j) t.P3[k][j] = (T)a.Ph_3[k * 3 + j];
            t.Psum3[k] = (T)a.Psum_3[k];
        }
        const double gh = p->opts.ao_gamma_hi, gl = p->opts.ao_gamma_lo;
        t.g_hi = (T)gh;
        t.g_hi1 = (T)(1.0 - gh);
        t.ig_hi = (T)(1.0 / gh);
        t.g3[0] = t.g3[2] = (T)(0.5 * (1.0 - gh) * (1.0 - gl));
        t.g3[1] = (T)((1.0 - gh) * gl);
        return t;
    } else {
        return make_tables<T, R>(p);
    }
}

// Schedule of the 2D kernel: strips as wide as the block allows (balanced
// widths), one CTA per resident slot, each CTA an equal share of the strips'
// rows (at least 8 rows, so the 5 warm-up y-face rows stay a minor cost).
inline Schedule schedule2d(int nx, int ny, int nt, int slots)
{
    Schedule s;
    const int wmax = nt - 5;
    s.nstrips = (nx + wmax - 1) / wmax;
    s.W = (nx + s.nstrips - 1) / s.nstrips;
    const long long rows = (long long)s.nstrips * ny;
    s.grid = (int)std::max(1LL, std::min<long long>(slots, rows / 8));
    s.H = (int)((rows + s.grid - 1) / s.grid);
    s.nseg = 0;
    return s;
}

template <typename T>
StageArgs<T> base_args(const gpweno_plan_s *p)
{
    StageArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; ++d) {
        a.n[d] = p->dims.n[d];
        a.per[d] = p->dims.bc_lo[d] == GPWENO_BC_PERIODIC ? 1 : 0;
        a.idx[d] = (T)(1.0 / p->dims.dx[d]);
    }
    a.flags = reinterpret_cast<int *>(p->ws + 3);
    a.cstride = p->ncell;
    a.P = nullptr;
    const int sd = p->dims.ndim - 1;   // the slab dimension: the slowest one
    a.ext[0] = p->dims.bc_lo[sd] == GPWENO_BC_EXTERNAL;
    a.ext[1] = p->dims.bc_hi[sd] == GPWENO_BC_EXTERNAL;
    a.slab_dim = (a.ext[0] || a.ext[1]) ? sd : -1;
    a.halo[0] = static_cast<const T *>(p->halo[0]);
    a.halo[1] = static_cast<const T *>(p->halo[1]);
    return a;
}

// Rows per CTA below which FP32 R = 2 grids take the three-CTA-per-SM build of the 2D kernel.
constexpr int kWideRows = 24;

// One launch of the 2D stage kernel built for MINB resident CTAs per SM: occupancy (queried
// once per instantiation), the one-wave schedule, the launch.
template <typename T, int R, int NT, int VAR, int MINB>
gpweno_status launch_stage2d(gpweno_plan p, StageArgs<T> a, const TablesFor<T, R, VAR> &tb, cudaStream_t st)
{
    const size_t smem = stage2d_smem_bytes<T, R, NT>();
    auto kern = stage2d_kernel<T, R, NT, VAR, MINB>;
    static int occ = 0;   // per instantiation: resident CTAs per SM
    if (!occ) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "stage2d smem attribute");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
        if (e != cudaSuccess || occ < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                          "stage2d occupancy");
    }
    Schedule s = schedule2d(a.n[0], a.n[1], NT, occ * p->num_sms);
    s.ctas_per_sm = occ;
    a.W = s.W;
    a.nstrips = s.nstrips;
    a.H = s.H;
    a.nseg = s.nseg;
    p->sched = s;
    cudaError_t e = launch_pdl(kern, s.grid, NT, smem, st, a, tb);
    if (e != cudaSuccess) return cuda_fail(e, "stage2d kernel launch");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
    return GPWENO_OK;
}

// VAR: the scheme variant (kVarMean: non-zero-mean smoothness indicators,
// kVarFdFlux: the FD-Flux form), a compile-time switch so that the default
// kernels keep their register budget.
template <typename T, int R, int VAR>
gpweno_status launch_stage_R(gpweno_plan p, const StageArgs<T> &a0, cudaStream_t st)
{
    StageArgs<T> a = a0;
    const TablesFor<T, R, VAR> tb = make_tables_var<T, R, VAR>(p);
    if (p->dims.ndim == 3) {
        // (1) xy-plane kernel: P = -(div_x/dx + div_y/dy)
        {
            constexpr int NT = kNTxy<T>;
            const size_t smem = stage2d_smem_bytes<T, R, NT, 5>();
            auto kern = plane3d_kernel<T, R, NT, VAR>;
            static int occ = 0;
            if (!occ) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return cuda_fail(e, "plane3d smem attribute");
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
                if (e != cudaSuccess || occ < 1)
                    return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "plane3d occupancy");
            }
            StageArgs<T> pa = a;
            const int wmax = NT - 5;
            pa.nstrips = (a.n[0] + wmax - 1) / wmax;
            pa.W = (a.n[0] + pa.nstrips - 1) / pa.nstrips;
            pa.mode = kModePartial;
            pa.out = const_cast<T *>(a.P);
            pa.rate = nullptr;
            const long long rows = (long long)pa.nstrips * a.n[1] * a.n[2];
            const int grid = (int)std::max(1LL, std::min<long long>((long long)occ * p->num_sms, rows / 8));
            cudaError_t e = launch_pdl(kern, grid, NT, smem, st, pa, tb);
            if (e != cudaSuccess) return cuda_fail(e, "plane3d kernel launch");
            count_launch(1);
        }
        // (2) z-marching kernel: L = P - div_z/dz and the stage update
        {
            constexpr int NT = kNTz;
            const size_t smem = stagez_smem_bytes<T, R, NT>();
            auto kern = stagez_kernel<T, R, NT, VAR>;
            static int occ = 0;
            if (!occ) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return cuda_fail(e, "stagez smem attribute");
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
                if (e != cudaSuccess || occ < 1)
                    return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "stagez occupancy");
            }
            const long long cols = ((long long)a.n[0] * a.n[1] + NT - 1) / NT * a.n[2];
            const int grid = (int)std::max(1LL, std::min<long long>((long long)occ * p->num_sms, cols / 8));
            cudaError_t e = launch_pdl(kern, grid, NT, smem, st, a, tb);
            if (e != cudaSuccess) return cuda_fail(e, "stagez kernel launch");
        }
    } else if (p->dims.ndim == 2) {
        constexpr int NT = kNTxy<T>;
        // FP32, default scheme (also with slab halos): the build for three CTAs per SM (more
        // registers per thread: R = 1/2/3 132/151/163 instead of 121/128/128) is faster where the
        // four-CTA schedule cannot fill four CTAs per SM (the grid is row-limited), and for
        // R = 2, whose four-CTA build is register-capped, where it leaves a CTA fewer than
        // kWideRows rows (three CTAs per SM: fewer, taller segments, fewer warm-up rows).
        // Measured on GB300 (same-box A/B, bitwise-identical results): R = 2 x1.10 at 512^2,
        // x1.05 at 768^2, x1.017 at 1024^2; R = 1 x1.14 and R = 3 x1.076 at 512^2.  Not taken
        // where it lost: R = 2 at 1536^2 (x0.995) and 4096^2 (x0.98), R = 1 at 1024^2 (x0.98),
        // R = 3 at 1024^2 (x0.986).
        constexpr bool kHasWide = std::is_same<T, float>::value && (VAR == 0 || VAR == kVarSlab);
        if constexpr (kHasWide) {
            const int slots4 = 512 / NT * p->num_sms;
            const Schedule s4 = schedule2d(a.n[0], a.n[1], NT, slots4);
            const long long rows = (long long)s4.nstrips * a.n[1];
            const bool row_limited = s4.grid < slots4;
            const bool short_segments = R == 2 && rows < (long long)kWideRows * s4.grid;
            if (row_limited || short_segments) {
                gpweno_status r = launch_stage2d<T, R, NT, VAR, 3>(p, a, tb, st);
                if (r != GPWENO_OK) return r;
                count_launch(1);
                return GPWENO_OK;
            }
        }
        gpweno_status r = launch_stage2d<T, R, NT, VAR, (sizeof(T) == 4 ? 512 : 256) / NT>(p, a, tb, st);
        if (r != GPWENO_OK) return r;
    } else {
        constexpr int NT = kNT1D;
        const size_t smem = stage1d_smem_bytes<T, R, NT>();
        auto kern = stage1d_kernel<T, R, NT, VAR>;
        a.nstrips = (a.n[0] + (NT - 5) - 1) / (NT - 5);
        a.W = (a.n[0] + a.nstrips - 1) / a.nstrips;
        a.H = 1;
        a.nseg = 1;
        cudaError_t e = launch_pdl(kern, a.nstrips, NT, smem, st, a, tb);
        if (e != cudaSuccess) return cuda_fail(e, "stage1d kernel launch");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

template <typename T, int VAR>
gpweno_status launch_stage_T(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    StageArgs<T> a = base_args<T>(p);
    a.U = static_cast<const T *>(io.U);
    a.U0 = static_cast<const T *>(io.U0);
    a.Din = static_cast<const T *>(io.Din);
    a.Dout = static_cast<T *>(io.Dout);
    a.Vout = static_cast<T *>(io.Vout);
    a.out = static_cast<T *>(io.out);
    a.P = static_cast<const T *>(io.P);
    a.lo = static_cast<T *>(io.lo);
    a.u0_is_stencil = io.U0 == io.U ? 1 : 0;
    a.b = (T)io.b;
    a.mode = io.mode;
    a.dt = io.dt;
    a.dt_dev = io.dt_dev;
    a.rate = io.want_rate ? p->ws : nullptr;
    switch (p->R) {
    case 1:
        if constexpr ((VAR & kVarAo) != 0) {
            set_error("GP-AO needs R = 2 or 3");
            return GPWENO_ERR_ARG;
        } else {
            return launch_stage_R<T, 1, VAR>(p, a, st);
        }
    case 2: return launch_stage_R<T, 2, VAR>(p, a, st);
    case 3: return launch_stage_R<T, 3, VAR>(p, a, st);
    default: set_error("R=%d not compiled", p->R); return GPWENO_ERR_ARG;
    }
}

template <typename T>
gpweno_status launch_max_rate_T(gpweno_plan p, const void *U, cudaStream_t st)
{
    StageArgs<T> a = base_args<T>(p);
    a.rate = p->ws;
    const int blocks = (int)std::min<long>((p->ncell + 255) / 256, 4L * p->num_sms);
    if (p->dims.ndim == 3)
        max_rate_kernel<T, 5><<<blocks, 256, 0, st>>>(static_cast<const T *>(U), p->ncell, a, (T)p->gamma);
    else if (p->dims.ndim == 2)
        max_rate_kernel<T, 4><<<blocks, 256, 0, st>>>(static_cast<const T *>(U), p->ncell, a, (T)p->gamma);
    else
        max_rate_kernel<T, 3><<<blocks, 256, 0, st>>>(static_cast<const T *>(U), p->ncell, a, (T)p->gamma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "max-rate kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

}  // namespace gpweno
