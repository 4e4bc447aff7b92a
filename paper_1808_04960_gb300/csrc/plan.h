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
};

}  // namespace gpweno

struct gpweno_plan_s {
    int R = 2;
    double ell = 12.0;
    gpweno_dims dims{};
    double gamma = 1.4;
    gpweno_opts opts{};
    gpweno::GpTables tab{};
    int device = 0;
    int num_sms = 0;
    long ncell = 0;
    // device workspace: [0..2] rate maxima (double bits), [3] flags
    unsigned long long *ws = nullptr;
    gpweno::Schedule sched;
    bool is_batch = false;
    // batch-only data
    std::vector<gpweno_plan> members;
    void *batch_dev = nullptr;     // device copy of per-instance descriptors
    size_t batch_bytes = 0;
    int batch_items = 0;
    int batch_grid = 0;
    std::vector<long> member_ncell;
};

namespace gpweno {

void set_error(const char *fmt, ...);
gpweno_status cuda_fail(cudaError_t e, const char *what);
void count_launch(int n);

// One stage launch (see StageArgs in stage.cuh for the meaning of each buffer).
struct StageIO {
    const void *U = nullptr;     // stencil state
    const void *U0 = nullptr;    // U^n at the output cells
    const void *Din = nullptr;   // previous increment
    void *Dout = nullptr;        // increment out (mode 1)
    void *Vout = nullptr;        // U^n + increment (mode 1)
    void *out = nullptr;         // RHS (mode 0) or U^{n+1} (mode 2)
    void *lo = nullptr;          // compensation remainder (mode 2)
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

// dispatch entry points implemented in stage_f32.cu / stage_f64.cu
gpweno_status launch_stage_f32(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_stage_f64(gpweno_plan p, const StageIO &io, cudaStream_t st);
gpweno_status launch_max_rate_f32(gpweno_plan p, const void *U, cudaStream_t st);
gpweno_status launch_max_rate_f64(gpweno_plan p, const void *U, cudaStream_t st);
gpweno_status launch_batch_stage_f32(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st);
gpweno_status launch_batch_stage_f64(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st);
gpweno_status build_batch_f32(gpweno_plan batch);
gpweno_status build_batch_f64(gpweno_plan batch);

}  // namespace gpweno
