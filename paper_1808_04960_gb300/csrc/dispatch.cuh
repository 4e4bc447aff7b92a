// Host-side launch of the stage kernels for one arithmetic type: table
// conversion, schedule (strip width, segment height, grid), kernel selection.
#pragma once
#include <algorithm>

#include "plan.h"
#include "stage.cuh"

namespace gpweno {

constexpr int kNT2D = 256;
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
        }
    for (int k = 0; k < S; ++k)
        for (int j = 0; j < (R + 2) / 2; ++j) t.Ph[k][j] = (T)p->tab.Ph[k * S + j];
    for (int m = 0; m < S; ++m) {
        t.gl[m] = (T)p->tab.gl[m];
        t.gr[m] = (T)p->tab.gr[m];
        t.sl1[m] = (T)p->tab.sl1[m];
        t.sr1[m] = (T)p->tab.sr1[m];
        t.Psum[m] = (T)p->tab.Psum[m];
    }
    t.eps = (T)p->opts.eps;
    t.gamma = (T)p->gamma;
    t.p = p->opts.p;
    t.flux = p->opts.flux_form;
    return t;
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
    return a;
}

// VAR: the scheme variant (kVarMean: non-zero-mean smoothness indicators,
// kVarFdFlux: the FD-Flux form), a compile-time switch so that the default
// kernels keep their register budget.
template <typename T, int R, int VAR>
gpweno_status launch_stage_R(gpweno_plan p, const StageArgs<T> &a0, cudaStream_t st)
{
    StageArgs<T> a = a0;
    const FaceTables<T, R> tb = make_tables<T, R>(p);
    if (p->dims.ndim == 3) {
        constexpr int NT = kNT2D;
        // (1) xy-plane kernel: P = -(div_x/dx + div_y/dy)
        {
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
            kern<<<grid, NT, smem, st>>>(pa, tb);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "plane3d kernel launch");
            count_launch(1);
        }
        // (2) z-marching kernel: L = P - div_z/dz and the stage update
        {
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
            kern<<<grid, NT, smem, st>>>(a, tb);
        }
    } else if (p->dims.ndim == 2) {
        constexpr int NT = kNT2D;
        const size_t smem = stage2d_smem_bytes<T, R, NT>();
        auto kern = stage2d_kernel<T, R, NT, VAR>;
        static int occ = 0;   // per instantiation: resident CTAs per SM
        if (!occ) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "stage2d smem attribute");
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
            if (e != cudaSuccess || occ < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                              "stage2d occupancy");
        }
        Schedule s = schedule2d(a.n[0], a.n[1], NT, occ * p->num_sms);
        a.W = s.W;
        a.nstrips = s.nstrips;
        a.H = s.H;
        a.nseg = s.nseg;
        p->sched = s;
        kern<<<s.grid, NT, smem, st>>>(a, tb);
    } else {
        constexpr int NT = kNT1D;
        const size_t smem = stage1d_smem_bytes<T, R, NT>();
        auto kern = stage1d_kernel<T, R, NT, VAR>;
        a.nstrips = (a.n[0] + (NT - 5) - 1) / (NT - 5);
        a.W = (a.n[0] + a.nstrips - 1) / a.nstrips;
        a.H = 1;
        a.nseg = 1;
        kern<<<a.nstrips, NT, smem, st>>>(a, tb);
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
    case 1: return launch_stage_R<T, 1, VAR>(p, a, st);
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
