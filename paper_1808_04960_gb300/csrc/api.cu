// C ABI of the GP-WENO library: plan lifetime, argument checks, the RK3 step
// sequence and error reporting.  Kernels live in stage_f32.cu / stage_f64.cu.
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "plan.h"

namespace gpweno {

static thread_local char g_err[512] = "";
static thread_local int g_launches = 0;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

gpweno_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return GPWENO_ERR_CUDA;
}

void count_launch(int n) { g_launches += n; }

void reset_launch_count() { g_launches = 0; }

__global__ void dt_from_rate_kernel(unsigned long long *rate, int ndim, double cfl, double *dt_dev)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int d = 0; d < ndim; ++d) {
            s += __longlong_as_double((long long)rate[d]);
            rate[d] = 0ull;
        }
        *dt_dev = cfl / s;
    }
}

}  // namespace gpweno

using namespace gpweno;

#define GPW_CHECK(x, what)                              \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

extern "C" {

void gpweno_default_opts(gpweno_opts *o)
{
    if (!o) return;
    o->sigma_over_dx = 3.0;
    o->eps = 1e-36;
    o->p = 2;
    o->dtype = GPWENO_F64;
    o->cfl = 0.0;
    o->flux_form = 0;
    o->beta_mean = 0;
    o->candidates = 0;
    o->scheme = 0;
    o->ao = 0;
    o->ao_gamma_hi = 0.85;
    o->ao_gamma_lo = 0.85;
}

const char *gpweno_last_error(void) { return g_err; }

int gpweno_last_launch_count(void) { return g_launches; }

gpweno_status gpweno_plan_create(gpweno_plan *out, int R, double ell_over_dx, const gpweno_dims *dims,
                                 double gamma_gas, const gpweno_opts *opts)
{
    if (!out || !dims) {
        set_error("gpweno_plan_create: null argument");
        return GPWENO_ERR_ARG;
    }
    *out = nullptr;
    gpweno_opts o;
    gpweno_default_opts(&o);
    if (opts) o = *opts;
    if (dims->ndim < 1 || dims->ndim > 3) {
        set_error("ndim=%d must be 1, 2 or 3", dims->ndim);
        return GPWENO_ERR_ARG;
    }
    if (!(gamma_gas > 1.0)) {
        set_error("gamma=%g must exceed 1", gamma_gas);
        return GPWENO_ERR_ARG;
    }
    if (o.dtype != GPWENO_F32 && o.dtype != GPWENO_F64) {
        set_error("dtype=%d invalid", o.dtype);
        return GPWENO_ERR_ARG;
    }
    if (o.p != 1 && o.p != 2) {
        set_error("p=%d must be 1 or 2", o.p);
        return GPWENO_ERR_ARG;
    }
    if (!(o.eps > 0.0) || (o.dtype == GPWENO_F32 && o.eps < 1.2e-38)) {
        set_error("eps=%g must be positive (and a normal FP32 number for dtype F32)", o.eps);
        return GPWENO_ERR_ARG;
    }
    if ((o.beta_mean != 0 && o.beta_mean != 1) || (o.candidates != 0 && o.candidates != 1)) {
        set_error("beta_mean=%d and candidates=%d must each be 0 or 1", o.beta_mean, o.candidates);
        return GPWENO_ERR_ARG;
    }
    if (o.ao != 0 && o.ao != 1) {
        set_error("ao=%d must be 0 or 1", o.ao);
        return GPWENO_ERR_ARG;
    }
    if (o.ao && ((R != 2 && R != 3) || o.scheme != 0 || o.candidates != 0)) {
        set_error("GP-AO needs R = 2 or 3, scheme = 0 and candidates = 0 (R=%d, scheme=%d, candidates=%d)", R,
                  o.scheme, o.candidates);
        return GPWENO_ERR_ARG;
    }
    if (o.ao && !(o.ao_gamma_hi > 0.0 && o.ao_gamma_hi < 1.0 && o.ao_gamma_lo > 0.0 && o.ao_gamma_lo < 1.0)) {
        set_error("ao_gamma_hi=%g and ao_gamma_lo=%g must lie in (0,1)", o.ao_gamma_hi, o.ao_gamma_lo);
        return GPWENO_ERR_ARG;
    }
    if (o.scheme != 0 && o.scheme != 1) {
        set_error("scheme=%d: 0 (FD-Prim) or 1 (FD-Flux)", o.scheme);
        return GPWENO_ERR_ARG;
    }
    if (o.scheme == 1 && o.flux_form != 0) {
        set_error("scheme=1 (FD-Flux) splits the fluxes itself; flux_form must be 0, got %d", o.flux_form);
        return GPWENO_ERR_ARG;
    }
    if (o.flux_form < 0 || o.flux_form > 2) {
        set_error("flux_form=%d: 0 (local Lax-Friedrichs), 1 (HLLC) or 2 (HLL)", o.flux_form);
        return GPWENO_ERR_ARG;
    }
    long ncell = 1;
    for (int d = 0; d < dims->ndim; ++d) {
        if (dims->n[d] < 1 || dims->n[d] > (1 << 24)) {
            set_error("n[%d]=%d out of range", d, dims->n[d]);
            return GPWENO_ERR_ARG;
        }
        if (!(dims->dx[d] > 0.0)) {
            set_error("dx[%d]=%g must be positive", d, dims->dx[d]);
            return GPWENO_ERR_ARG;
        }
        bool plo = dims->bc_lo[d] == GPWENO_BC_PERIODIC, phi = dims->bc_hi[d] == GPWENO_BC_PERIODIC;
        if (plo != phi) {
            set_error("dimension %d: periodic must be set on both sides or neither", d);
            return GPWENO_ERR_ARG;
        }
        if ((dims->bc_lo[d] != 0 && dims->bc_lo[d] != 1) || (dims->bc_hi[d] != 0 && dims->bc_hi[d] != 1)) {
            set_error("dimension %d: unknown boundary condition", d);
            return GPWENO_ERR_ARG;
        }
        ncell *= dims->n[d];
    }
    if (ncell > (1L << 31)) {
        set_error("grid of %ld cells exceeds the 2^31-cell limit of the library", ncell);
        return GPWENO_ERR_ARG;
    }
    gpweno_plan p = new (std::nothrow) gpweno_plan_s();
    if (!p) {
        set_error("out of host memory");
        return GPWENO_ERR_ARG;
    }
    p->R = R;
    p->ell = ell_over_dx;
    p->dims = *dims;
    for (int d = dims->ndim; d < 3; ++d) {
        p->dims.n[d] = 1;
        p->dims.dx[d] = 1.0;
        p->dims.bc_lo[d] = p->dims.bc_hi[d] = GPWENO_BC_OUTFLOW;
    }
    p->gamma = gamma_gas;
    p->opts = o;
    p->ncell = ncell;
    char err[256];
    int rc = gp_precompute(R, ell_over_dx, o.sigma_over_dx, &p->tab, err, sizeof(err), o.candidates, o.scheme);
    if (!rc && o.ao) rc = ao_precompute(R, ell_over_dx, o.sigma_over_dx, &p->ao, err, sizeof(err));
    if (rc) {
        set_error("%s", err);
        delete p;
        return rc == 1 ? GPWENO_ERR_ARG : GPWENO_ERR_PRECOMPUTE;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->ws, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->ws, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        if (p->ws) cudaFree(p->ws);
        delete p;
        return cuda_fail(e, "gpweno_plan_create");
    }
    *out = p;
    return GPWENO_OK;
}

gpweno_status gpweno_plan_destroy(gpweno_plan p)
{
    if (!p) return GPWENO_OK;
    if (p->ws) cudaFree(p->ws);
    if (p->batch_inst_dev) cudaFree(p->batch_inst_dev);
    if (p->batch_inst_host) cudaFreeHost(p->batch_inst_host);
    if (p->batch_segs_dev) cudaFree(p->batch_segs_dev);
    if (p->batch_cta_dev) cudaFree(p->batch_cta_dev);
    delete p;
    return GPWENO_OK;
}

gpweno_status gpweno_plan_tables(gpweno_plan p, double *w_m, double *gam, double *P, double *w_big)
{
    if (!p || p->is_batch) {
        set_error("gpweno_plan_tables: invalid plan");
        return GPWENO_ERR_ARG;
    }
    const int S = p->R + 1;
    if (w_m) std::memcpy(w_m, p->tab.wl, sizeof(double) * S * S);
    if (gam) std::memcpy(gam, p->tab.gl, sizeof(double) * S);
    if (P) std::memcpy(P, p->tab.P, sizeof(double) * S * S);
    if (w_big) std::memcpy(w_big, p->tab.wbig_l, sizeof(double) * (2 * p->R + 1));
    return GPWENO_OK;
}

gpweno_status gpweno_gp_tables(int R, double ell_over_dx, double sigma_over_dx, int candidates, int scheme,
                               double *w_m, double *gam, double *P, double *w_big, double *w_m_r, double *gam_r)
{
    GpTables t;
    char err[256];
    if ((candidates != 0 && candidates != 1) || (scheme != 0 && scheme != 1)) {
        set_error("candidates=%d and scheme=%d must each be 0 or 1", candidates, scheme);
        return GPWENO_ERR_ARG;
    }
    int rc = gp_precompute(R, ell_over_dx, sigma_over_dx, &t, err, sizeof(err), candidates, scheme);
    if (rc) {
        set_error("%s", err);
        return rc == 1 ? GPWENO_ERR_ARG : GPWENO_ERR_PRECOMPUTE;
    }
    const int S = R + 1;
    if (w_m) std::memcpy(w_m, t.wl, sizeof(double) * S * S);
    if (gam) std::memcpy(gam, t.gl, sizeof(double) * S);
    if (P) std::memcpy(P, t.P, sizeof(double) * S * S);
    if (w_big) std::memcpy(w_big, t.wbig_l, sizeof(double) * (2 * R + 1));
    if (w_m_r) std::memcpy(w_m_r, t.wr, sizeof(double) * S * S);
    if (gam_r) std::memcpy(gam_r, t.gr, sizeof(double) * S);
    return GPWENO_OK;
}

gpweno_status gpweno_ao_tables(int R, double ell_over_dx, double sigma_over_dx, double *w_hi, double *w_lo,
                               double *w3, double *P_hi, double *P_lo, double *P_3)
{
    AoTables t;
    char err[256];
    GpTables g;
    int rc = gp_precompute(R, ell_over_dx, sigma_over_dx, &g, err, sizeof(err));
    if (!rc) rc = ao_precompute(R, ell_over_dx, sigma_over_dx, &t, err, sizeof(err));
    if (rc) {
        set_error("%s", err);
        return rc == 1 ? GPWENO_ERR_ARG : GPWENO_ERR_PRECOMPUTE;
    }
    const int nh = 2 * R + 1, nl = 2 * R - 1;
    if (w_hi) {
        std::memcpy(w_hi, t.w_hi_l, sizeof(double) * nh);
        std::memcpy(w_hi + nh, t.w_hi_r, sizeof(double) * nh);
    }
    if (w_lo && R == 3) {
        std::memcpy(w_lo, t.w_lo_l, sizeof(double) * nl);
        std::memcpy(w_lo + nl, t.w_lo_r, sizeof(double) * nl);
    }
    if (w3) {
        std::memcpy(w3, t.w3_l, sizeof(double) * 9);
        std::memcpy(w3 + 9, t.w3_r, sizeof(double) * 9);
    }
    if (P_hi) std::memcpy(P_hi, t.P_hi, sizeof(double) * nh * nh);
    if (P_lo && R == 3) std::memcpy(P_lo, t.P_lo, sizeof(double) * nl * nl);
    if (P_3) std::memcpy(P_3, t.P_3, sizeof(double) * 9);
    return GPWENO_OK;
}

}  // extern "C"

static gpweno_status launch_stage(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    return p->opts.dtype == GPWENO_F32 ? launch_stage_f32(p, io, st) : launch_stage_f64(p, io, st);
}

namespace gpweno {

gpweno_status rk3_sequence(gpweno_plan p, void *U, void *D, void *V1, void *V2, void *lo, double dt,
                           const double *dt_dev, bool want_rate, cudaStream_t st)
{
    gpweno_status s;
    StageIO io;
    io.dt = dt;
    io.dt_dev = dt_dev;
    // D_1 = dt L(U^n), V_1 = U^n + D_1   (3D: the x+y part of L goes through the
    // buffer the stage update overwrites next: V1, V2, then the dead V1)
    io.P = V1;
    io.U = U;
    io.U0 = U;
    io.Dout = D;
    io.Vout = V1;
    io.b = 1.0;
    io.mode = 1;
    if ((s = launch_stage(p, io, st)) != GPWENO_OK) return s;
    // D_2 = 1/4 (D_1 + dt L(V_1)), V_2 = U^n + D_2
    io.U = V1;
    io.Din = D;
    io.Vout = V2;
    io.P = V2;
    io.b = 0.25;
    if ((s = launch_stage(p, io, st)) != GPWENO_OK) return s;
    // U^{n+1} = U^n + 2/3 (D_2 + dt L(V_2)), compensated with lo
    io.U = V2;
    io.Dout = nullptr;
    io.Vout = nullptr;
    io.P = V1;
    io.out = U;
    io.lo = lo;
    io.b = 2.0 / 3.0;
    io.mode = 2;
    io.want_rate = want_rate;
    return launch_stage(p, io, st);
}

}  // namespace gpweno

static bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

extern "C" {

gpweno_status gpweno_rhs(gpweno_plan p, const void *U, void *dUdt, void *stream)
{
    g_launches = 0;
    if (!p || p->is_batch || !U || !dUdt) {
        set_error("gpweno_rhs: invalid argument");
        return GPWENO_ERR_ARG;
    }
    if (U == dUdt || !aligned16(U) || !aligned16(dUdt)) {
        set_error("gpweno_rhs: U and dUdt must be distinct 16-byte aligned buffers");
        return GPWENO_ERR_ARG;
    }
    StageIO io;
    io.U = U;
    io.out = dUdt;
    io.P = dUdt;
    io.mode = 0;
    return launch_stage(p, io, (cudaStream_t)stream);
}

gpweno_status gpweno_rk3_step(gpweno_plan p, void *U, void *scratch, double dt, void *dt_dev, void *stream)
{
    g_launches = 0;
    if (!p || p->is_batch || !U || !scratch) {
        set_error("gpweno_rk3_step: invalid argument");
        return GPWENO_ERR_ARG;
    }
    if (!aligned16(U) || !aligned16(scratch)) {
        set_error("gpweno_rk3_step: buffers must be 16-byte aligned");
        return GPWENO_ERR_ARG;
    }
    if (!dt_dev && !(dt > 0.0)) {
        set_error("gpweno_rk3_step: dt=%g must be positive", dt);
        return GPWENO_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = p->opts.dtype == GPWENO_F32 ? 4 : 8;
    const size_t bytes = esz * (size_t)(p->dims.ndim + 2) * (size_t)p->ncell;
    char *base = static_cast<char *>(scratch);
    const double *dtp = static_cast<const double *>(dt_dev);
    const bool cfl = dt_dev && p->opts.cfl > 0.0;
    gpweno_status s = rk3_sequence(p, U, base, base + bytes, base + 2 * bytes, base + 3 * bytes, dt, dtp, cfl, st);
    if (s != GPWENO_OK) return s;
    if (cfl) {
        dt_from_rate_kernel<<<1, 32, 0, st>>>(p->ws, p->dims.ndim, p->opts.cfl, static_cast<double *>(dt_dev));
        GPW_CHECK(cudaGetLastError(), "dt kernel launch");
        count_launch(1);
    }
    return GPWENO_OK;
}

gpweno_status gpweno_cfl_dt(gpweno_plan p, const void *U, double cfl, void *dt_dev, void *stream)
{
    g_launches = 0;
    if (!p || p->is_batch || !U || !dt_dev || !(cfl > 0.0)) {
        set_error("gpweno_cfl_dt: invalid argument");
        return GPWENO_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gpweno_status s =
        p->opts.dtype == GPWENO_F32 ? launch_max_rate_f32(p, U, st) : launch_max_rate_f64(p, U, st);
    if (s != GPWENO_OK) return s;
    dt_from_rate_kernel<<<1, 32, 0, st>>>(p->ws, p->dims.ndim, cfl, static_cast<double *>(dt_dev));
    GPW_CHECK(cudaGetLastError(), "dt kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

gpweno_status gpweno_flags(gpweno_plan p, int *nonphysical)
{
    if (!p || !nonphysical) {
        set_error("gpweno_flags: invalid argument");
        return GPWENO_ERR_ARG;
    }
    GPW_CHECK(cudaDeviceSynchronize(), "gpweno_flags: earlier launch failed");
    unsigned long long f = 0;
    GPW_CHECK(cudaMemcpy(&f, p->ws + 3, sizeof(f), cudaMemcpyDeviceToHost), "gpweno_flags: read");
    GPW_CHECK(cudaMemset(p->ws + 3, 0, sizeof(f)), "gpweno_flags: clear");
    *nonphysical = (f & 1ull) ? 1 : 0;
    return GPWENO_OK;
}

gpweno_status gpweno_plan_batch(gpweno_plan *out, const gpweno_plan *plans, int n, const char *tune_cache)
{
    if (!out || !plans || n < 1) {
        set_error("gpweno_plan_batch: need an output pointer and at least one plan");
        return GPWENO_ERR_ARG;
    }
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        gpweno_plan p = plans[k];
        if (!p || p->is_batch || p->dims.ndim != 2) {
            set_error("gpweno_plan_batch: plan %d is not a 2D single-grid plan", k);
            return GPWENO_ERR_ARG;
        }
        if (p->opts.beta_mean || p->opts.scheme || p->opts.ao) {
            set_error("gpweno_plan_batch: plan %d uses beta_mean, scheme = 1 or ao, which batches do not support", k);
            return GPWENO_ERR_ARG;
        }
        if (p->opts.dtype != plans[0]->opts.dtype || p->device != plans[0]->device) {
            set_error("gpweno_plan_batch: plan %d differs in dtype or device from plan 0", k);
            return GPWENO_ERR_ARG;
        }
    }
    gpweno_plan b = new (std::nothrow) gpweno_plan_s();
    if (!b) {
        set_error("out of host memory");
        return GPWENO_ERR_ARG;
    }
    b->is_batch = true;
    b->members.assign(plans, plans + n);
    b->opts = plans[0]->opts;
    b->device = plans[0]->device;
    b->num_sms = plans[0]->num_sms;
    b->dims.ndim = 2;
    if (tune_cache) b->batch_tune_path = tune_cache;
    cudaError_t e = cudaMalloc(&b->ws, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->ws, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        gpweno_plan_destroy(b);
        return cuda_fail(e, "gpweno_plan_batch workspace");
    }
    gpweno_status s = b->opts.dtype == GPWENO_F32 ? build_batch_f32(b) : build_batch_f64(b);
    if (s != GPWENO_OK) {
        gpweno_plan_destroy(b);
        return s;
    }
    *out = b;
    return GPWENO_OK;
}

gpweno_status gpweno_batch_rk3_step(gpweno_plan b, void *const *U, void *const *scratch, const void *dt_dev,
                                    void *stream)
{
    g_launches = 0;
    if (!b || !b->is_batch || !U || !scratch || !dt_dev) {
        set_error("gpweno_batch_rk3_step: invalid argument");
        return GPWENO_ERR_ARG;
    }
    const int n = (int)b->members.size();
    for (int k = 0; k < n; ++k)
        if (!U[k] || !scratch[k] || !aligned16(U[k]) || !aligned16(scratch[k])) {
            set_error("gpweno_batch_rk3_step: buffers of instance %d missing or not 16-byte aligned", k);
            return GPWENO_ERR_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const double *dt = static_cast<const double *>(dt_dev);
    for (int stage = 0; stage < 3; ++stage) {
        gpweno_status s = b->opts.dtype == GPWENO_F32 ? launch_batch_stage_f32(b, stage, U, scratch, dt, st)
                                                      : launch_batch_stage_f64(b, stage, U, scratch, dt, st);
        if (s != GPWENO_OK) return s;
    }
    return GPWENO_OK;
}

int gpweno_batch_info(gpweno_plan b, int *block, int *ctas_per_sm, int *grid, int *segments,
                      unsigned long long *signature)
{
    if (!b || !b->is_batch) return GPWENO_ERR_ARG;
    if (block) *block = b->batch_nt;
    if (ctas_per_sm) *ctas_per_sm = b->batch_ctas_per_sm;
    if (grid) *grid = b->batch_grid;
    if (segments) *segments = b->batch_nseg;
    if (signature) *signature = b->batch_signature;
    return GPWENO_OK;
}

}  // extern "C"
