// Batched 2D stepping: one launch per SSP-RK3 stage for many independent
// instances of uneven size, radius R and length scales.
//
// The host flattens every instance into strips (as the single-instance
// kernel does) and cuts the strips' rows into segments so that each CTA share
// (several per resident slot) gets an equal part of the estimated cost (face work grows with R and with the
// number of 32-lane warps a strip keeps busy; every segment pays five
// warm-up y-face rows).  A CTA walks its contiguous run of segments and, per
// segment, dispatches on the instance's R to the same segment routine the
// single-instance kernel uses.  Weight tables are deduplicated on the host
// (instances with the same R, l/dx, sigma/dx, gamma share one set) and travel
// in a __grid_constant__ kernel parameter.
#pragma once
#include "stage.cuh"

namespace gpweno {

constexpr int kBatchMaxSets = 12;   // distinct table sets per radius in one batch

template <typename T>
struct BatchTables {
    FaceTables<T, 1> t1[kBatchMaxSets];
    FaceTables<T, 2> t2[kBatchMaxSets];
    FaceTables<T, 3> t3[kBatchMaxSets];
};

template <typename T>
struct BatchInst {
    const T *U;      // U^n (updated in place by the last stage)
    T *D;            // increment
    T *V1;           // U^n + D_1
    T *V2;           // U^n + D_2
    T *lo;           // compensation remainder
    int n[2];
    int per[2];
    T idx[2];
    int R;
    int tab;         // table set index for this R
    int W;           // strip width
    int nstrips;
};

struct BatchSeg {
    int inst, strip, y0, y1;
};

template <typename T, int NT>
constexpr size_t batch_smem_bytes()
{
    // the largest radius sets the ring size
    return stage2d_smem_bytes<T, 3, NT>();
}

// 512 (FP32) or 256 (FP64) resident threads per SM at most 128 / 255 registers each
template <typename T, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 512 : 256) / NT)
    batch_stage_kernel(const BatchInst<T> *__restrict__ inst, const BatchSeg *__restrict__ segs,
                       const int *__restrict__ cta_start, int stage, const double *__restrict__ dt_dev, int *flags,
                       const __grid_constant__ BatchTables<T> bt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    T rmx = T(0), rmy = T(0);
    bool ok = true;
    // per-segment arguments live in shared memory (filled by thread 0), which
    // keeps them out of the registers the face evaluation needs
    __shared__ StageArgs<T> sa;
    __shared__ BatchSeg ssg;
    __shared__ int sR, stab;
    __shared__ T sdt;
    const int k0 = cta_start[blockIdx.x], k1 = cta_start[blockIdx.x + 1];
    for (int k = k0; k < k1; ++k) {
        if (threadIdx.x == 0) {
            const BatchSeg sg = segs[k];
            const BatchInst<T> &I = inst[sg.inst];
            StageArgs<T> a;
            a.n[0] = I.n[0];
            a.n[1] = I.n[1];
            a.n[2] = 1;
            a.per[0] = I.per[0];
            a.per[1] = I.per[1];
            a.per[2] = 0;
            a.idx[0] = I.idx[0];
            a.idx[1] = I.idx[1];
            a.idx[2] = T(1);
            a.dt_dev = nullptr;
            a.dt = 0.0;
            a.rate = nullptr;
            a.flags = flags;
            a.W = I.W;
            a.nstrips = I.nstrips;
            a.H = 0;
            a.nseg = 0;
            a.U0 = I.U;
            a.out = nullptr;
            a.lo = nullptr;
            a.Dout = nullptr;
            a.Vout = nullptr;
            if (stage == 0) {
                a.U = I.U;
                a.Din = nullptr;
                a.Dout = I.D;
                a.Vout = I.V1;
                a.b = T(1);
                a.mode = kModeIncrement;
                a.u0_is_stencil = 1;
            } else if (stage == 1) {
                a.U = I.V1;
                a.Din = I.D;
                a.Dout = I.D;
                a.Vout = I.V2;
                a.b = T(0.25);
                a.mode = kModeIncrement;
                a.u0_is_stencil = 0;
            } else {
                a.U = I.V2;
                a.Din = I.D;
                a.out = const_cast<T *>(I.U);
                a.lo = I.lo;
                a.b = T(2.0 / 3.0);
                a.mode = kModeFinal;
                a.u0_is_stencil = 0;
            }
            a.cstride = (long)I.n[0] * I.n[1];
            a.P = nullptr;
            a.slab_dim = -1;   // batch instances have no external sides
            a.ext[0] = a.ext[1] = 0;
            a.halo[0] = a.halo[1] = nullptr;
            sa = a;
            ssg = sg;
            sR = I.R;
            stab = I.tab;
            sdt = (T)dt_dev[sg.inst];
        }
        __syncthreads();
        const BatchSeg sg = ssg;
        const T dt = sdt;
        const int tab = stab;
        // FP32: the two-site row loop and interleaved layout of the single-instance kernel (no
        // spills with all three radii in one kernel); FP64 keeps the one-site loop, whose smaller
        // code spills less at 255 registers
        constexpr bool kOneSite = sizeof(T) == 8;
        switch (sR) {
        case 1: stage2d_segment<T, 1, NT, 4, 0, kOneSite>(sa, bt.t1[tab], sg.strip, sg.y0, sg.y1, smem, dt, rmx, rmy, ok); break;
        case 2: stage2d_segment<T, 2, NT, 4, 0, kOneSite>(sa, bt.t2[tab], sg.strip, sg.y0, sg.y1, smem, dt, rmx, rmy, ok); break;
        default: stage2d_segment<T, 3, NT, 4, 0, kOneSite>(sa, bt.t3[tab], sg.strip, sg.y0, sg.y1, smem, dt, rmx, rmy, ok); break;
        }
        // the segment ends with a barrier, so thread 0 may overwrite the shared arguments
    }
    if (__any_sync(0xffffffffu, !ok) && (threadIdx.x & 31) == 0) atomicOr(flags, 1);
}

}  // namespace gpweno
