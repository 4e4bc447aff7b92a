// Internal plan definition shared by the host translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gpweno.h"
#include "gp_precompute.h"

namespace gpweno {

struct Schedule {
    int W = 0, nstrips = 0, H = 0, nseg = 0, grid = 0;
    int ctas_per_sm = 0;   // resident CTAs per SM of the kernel build the launch used
};

}  // namespace gpweno

struct gpweno_plan_s {
    int R = 2;
    double ell = 12.0;
    gpweno_dims dims{};
    double gamma = 1.4;
    gpweno_opts opts{};
    gpweno::GpTables tab{};
    gpweno::AoTables ao{};                  // GP-AO tables when opts.ao = 1
    int device = 0;
    int num_sms = 0;
    long ncell = 0;
    // device workspace: [0..2] rate maxima (double bits), [3] flags
    unsigned long long *ws = nullptr;
    gpweno::Schedule sched;
    const void *halo[2] = {nullptr, nullptr};   // halo buffers of external sides (gpweno_set_halo)
    bool is_batch = false;
    // batch-only data
    std::vector<gpweno_plan> members;
    int batch_nt = 256;                     // block size of the batch kernel
    int batch_ctas_per_sm = 2;              // resident CTAs per SM the schedule assumes
    int batch_wcap = 0;                     // widest strip (columns)
    int batch_min_rows = 8;                 // fewest rows of a segment that does not end its strip
    int batch_oversub = 1;                  // CTA shares per resident slot
    int batch_grid = 0;                     // CTAs per launch
    int batch_nseg = 0;                     // segments in the schedule
    unsigned long long batch_signature = 0; // hash of the instance list (tuning-cache key)
    std::string batch_tune_path;            // tuning cache file (may be empty)
    std::vector<unsigned char> batch_tables;   // BatchTables<T> bytes (kernel parameter)
    std::vector<int> member_tab;            // table set index per instance
    void *batch_inst_dev = nullptr;         // BatchInst<T>[n]
    void *batch_inst_host = nullptr;        // pinned staging of the same
    void *batch_segs_dev = nullptr;         // BatchSeg[nseg]
    void *batch_cta_dev = nullptr;          // int[grid+1]
    std::vector<const void *> batch_last_ptrs;  // U/scratch pointers of the last upload
};

namespace gpweno {

void set_error(const char *fmt, ...);
gpweno_status cuda_fail(cudaError_t e, const char *what);
void count_launch(int n);
void reset_launch_count();

// One stage launch (see StageArgs in stage.cuh for the meaning of each buffer).
struct StageIO {
    const void *U = nullptr;     // stencil state
    const void *U0 = nullptr;    // U^n at the output cells
    const void *Din = nullptr;   // previous increment
    void *Dout = nullptr;        // increment out (mode 1)
    void *Vout = nullptr;        // U^n + increment (mode 1)
    void *out = nullptr;         // RHS (mode 0) or U^{n+1} (mode 2)
    void *lo = nullptr;          // compensation remainder (mode 2)
    void *P = nullptr;           // 3D: buffer for the x+y part of L (read back cell by cell)
    double b = 1.0;
    int mode = 0;
    double dt = 0.0;
    const double *dt_dev = nullptr;
    bool want_rate = false;
};

// The three stage launches of one SSP-RK3 step on caller buffers:
// D, V1, V2 are state-sized stage buffers; lo is the compensation remainder (or null).
gpweno_status rk3_sequence(gpweno_plan p, void *U, void *D, void *V1, void *V2, void *lo, double dt,
                           const double *dt_dev, bool want_rate, cudaStream_t st);
// Whether the plan has a GPWENO_BC_EXTERNAL side (slab decomposition).
bool has_external_side(const gpweno_plan_s *p);

// dispatch entry points implemented in stage_f32.cu / stage_f64.cu
gpweno_status launch_stage_f32(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64(gpweno_plan p, const StageIO &io, cudaStream_t st);
// variants (kVarMean = 1 non-zero-mean beta, kVarFdFlux = 2 FD-Flux, kVarAo = 4 GP-AO):
// 1, 2, 3 = FD-Flux with mean, 4 = AO, 5 = AO with mean
gpweno_status launch_stage_f32_var1(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f32_var2(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f32_var3(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f32_var4(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f32_var5(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var1(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var2(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var3(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var4(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var5(gpweno_plan p, const StageIO &io, cudaStream_t st);
// grids with an external (halo) side: kVarSlab = 8
gpweno_status launch_stage_f32_var8(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64_var8(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_max_rate_f32(gpweno_plan p, const void *U, cudaStream_t st);
gpweno_status launch_max_rate_f64(gpweno_plan p, const void *U, cudaStream_t st);
gpweno_status launch_batch_stage_f32(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st);
gpweno_status launch_batch_stage_f64(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st);
gpweno_status build_batch_f32(gpweno_plan batch);
gpweno_status build_batch_f64(gpweno_plan batch);

}  // namespace gpweno
