// C ABI of the GP-WENO library: plan lifetime, argument checks, the RK3 step
// sequence and error reporting.  Kernels live in stage_f32.cu / stage_f64.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "plan.h"
#include "trace.h"

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
        if (dims->bc_lo[d] < 0 || dims->bc_lo[d] > 2 || dims->bc_hi[d] < 0 || dims->bc_hi[d] > 2) {
            set_error("dimension %d: unknown boundary condition", d);
            return GPWENO_ERR_ARG;
        }
        const bool ext = dims->bc_lo[d] == GPWENO_BC_EXTERNAL || dims->bc_hi[d] == GPWENO_BC_EXTERNAL;
        if (ext && d != dims->ndim - 1) {
            set_error("dimension %d: external (halo) sides are allowed on the slowest dimension %d only", d,
                      dims->ndim - 1);
            return GPWENO_ERR_ARG;
        }
        if (ext && (o.beta_mean || o.scheme || o.ao)) {
            set_error("external (halo) sides are supported by the default scheme (beta_mean = 0, scheme = 0, ao = 0)");
            return GPWENO_ERR_ARG;
        }
        if (ext && dims->n[d] < R + 3) {
            set_error("dimension %d: a slab with external sides needs at least R+3 = %d cells, has %d", d, R + 3,
                      dims->n[d]);
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

// Buffers and weights of stage k of the increment-form SSP-RK3 step.  The 3D
// x+y part of L goes through the buffer the stage update overwrites next: V1,
// V2, then the dead V1.
static StageIO stage_io(int k, void *U, void *D, void *V1, void *V2, void *lo, double dt, const double *dt_dev,
                        bool want_rate)
{
    StageIO io;
    io.dt = dt;
    io.dt_dev = dt_dev;
    io.U0 = U;
    if (k == 0) {          // D_1 = dt L(U^n), V_1 = U^n + D_1
        io.P = V1;
        io.U = U;
        io.Dout = D;
        io.Vout = V1;
        io.b = 1.0;
        io.mode = 1;
    } else if (k == 1) {   // D_2 = 1/4 (D_1 + dt L(V_1)), V_2 = U^n + D_2
        io.P = V2;
        io.U = V1;
        io.Din = D;
        io.Dout = D;
        io.Vout = V2;
        io.b = 0.25;
        io.mode = 1;
    } else {               // U^{n+1} = U^n + 2/3 (D_2 + dt L(V_2)), compensated with lo
        io.P = V1;
        io.U = V2;
        io.Din = D;
        io.out = U;
        io.lo = lo;
        io.b = 2.0 / 3.0;
        io.mode = 2;
        io.want_rate = want_rate;
    }
    return io;
}

gpweno_status rk3_sequence(gpweno_plan p, void *U, void *D, void *V1, void *V2, void *lo, double dt,
                           const double *dt_dev, bool want_rate, cudaStream_t st)
{
    for (int k = 0; k < 3; ++k) {
        TraceRange tr(stage_range_name(k));
        gpweno_status s = launch_stage(p, stage_io(k, U, D, V1, V2, lo, dt, dt_dev, want_rate), st);
        if (s != GPWENO_OK) return s;
    }
    return GPWENO_OK;
}

bool has_external_side(const gpweno_plan_s *p)
{
    const int sd = p->dims.ndim - 1;
    return p->dims.bc_lo[sd] == GPWENO_BC_EXTERNAL || p->dims.bc_hi[sd] == GPWENO_BC_EXTERNAL;
}

// The halo buffers an external side needs are registered.
static gpweno_status check_halo(const gpweno_plan_s *p, const char *what)
{
    const int sd = p->dims.ndim - 1;
    if ((p->dims.bc_lo[sd] == GPWENO_BC_EXTERNAL && !p->halo[0]) ||
        (p->dims.bc_hi[sd] == GPWENO_BC_EXTERNAL && !p->halo[1])) {
        set_error("%s: the plan has external sides but no halo buffer was registered (gpweno_set_halo)", what);
        return GPWENO_ERR_ARG;
    }
    return GPWENO_OK;
}

// Copy the first and last G layers of a state along the slab dimension into
// the halo layout [nc][G][layer].
template <typename T>
__global__ void halo_pack_kernel(const T *__restrict__ s, T *lo, T *hi, long layer, int G, int n, int nc, long cstride)
{
    const long per_side = (long)nc * G * layer, block = (long)G * layer;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 2 * per_side; i += (long)gridDim.x * blockDim.x) {
        const int side = i >= per_side ? 1 : 0;
        T *dst = side ? hi : lo;
        if (!dst) continue;
        const long j = i - side * per_side;
        const long c = j / block, r = j - c * block;
        dst[j] = s[c * cstride + (side ? (long)(n - G) * layer : 0L) + r];
    }
}

// Copy the plan's rate maxima out and clear them.
__global__ void rate_export_kernel(unsigned long long *ws, unsigned long long *out)
{
    if (threadIdx.x < 3) {
        out[threadIdx.x] = ws[threadIdx.x];
        ws[threadIdx.x] = 0ull;
    }
}

// dt = cfl / sum_d rate_d from a caller's (reduced) rate maxima.
__global__ void dt_from_rates_kernel(const unsigned long long *rate, int ndim, double cfl, double *dt_dev)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int d = 0; d < ndim; ++d) s += __longlong_as_double((long long)rate[d]);
        *dt_dev = cfl / s;
    }
}

}  // namespace gpweno

static bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

extern "C" {

gpweno_status gpweno_rhs(gpweno_plan p, const void *U, void *dUdt, void *stream)
{
    TraceRange tr("gpweno_rhs");
    g_launches = 0;
    if (!p || p->is_batch || !U || !dUdt) {
        set_error("gpweno_rhs: invalid argument");
        return GPWENO_ERR_ARG;
    }
    if (U == dUdt || !aligned16(U) || !aligned16(dUdt)) {
        set_error("gpweno_rhs: U and dUdt must be distinct 16-byte aligned buffers");
        return GPWENO_ERR_ARG;
    }
    gpweno_status s = check_halo(p, "gpweno_rhs");
    if (s != GPWENO_OK) return s;
    StageIO io;
    io.U = U;
    io.out = dUdt;
    io.P = dUdt;
    io.mode = 0;
    return launch_stage(p, io, (cudaStream_t)stream);
}

gpweno_status gpweno_set_halo(gpweno_plan p, const void *recv_lo, const void *recv_hi)
{
    if (!p || p->is_batch || !has_external_side(p)) {
        set_error("gpweno_set_halo: needs a single-grid plan with an external side");
        return GPWENO_ERR_ARG;
    }
    const int sd = p->dims.ndim - 1;
    const bool elo = p->dims.bc_lo[sd] == GPWENO_BC_EXTERNAL, ehi = p->dims.bc_hi[sd] == GPWENO_BC_EXTERNAL;
    if ((elo && (!recv_lo || !aligned16(recv_lo))) || (ehi && (!recv_hi || !aligned16(recv_hi)))) {
        set_error("gpweno_set_halo: every external side needs a 16-byte aligned halo buffer");
        return GPWENO_ERR_ARG;
    }
    p->halo[0] = elo ? recv_lo : nullptr;
    p->halo[1] = ehi ? recv_hi : nullptr;
    return GPWENO_OK;
}

gpweno_status gpweno_halo_pack(gpweno_plan p, const void *state, void *send_lo, void *send_hi, void *stream)
{
    TraceRange tr("gpweno_halo_pack");
    g_launches = 0;
    const uintptr_t esz = p && p->opts.dtype == GPWENO_F32 ? 4 : 8;
    if (!p || p->is_batch || !state || (reinterpret_cast<uintptr_t>(state) % esz) != 0 ||
        (reinterpret_cast<uintptr_t>(send_lo) % esz) != 0 || (reinterpret_cast<uintptr_t>(send_hi) % esz) != 0) {
        set_error("gpweno_halo_pack: invalid argument (null plan or state, or a buffer not aligned to its element)");
        return GPWENO_ERR_ARG;
    }
    const int sd = p->dims.ndim - 1, G = p->R + 3, n = p->dims.n[sd];
    if (n < G) {
        set_error("gpweno_halo_pack: the slowest dimension has %d cells, fewer than G = %d", n, G);
        return GPWENO_ERR_ARG;
    }
    if (!send_lo && !send_hi) return GPWENO_OK;
    const long layer = p->ncell / n;
    const long total = 2L * (p->dims.ndim + 2) * G * layer;
    const int blocks = (int)std::min<long>((total + 255) / 256, 8L * p->num_sms);
    cudaStream_t st = (cudaStream_t)stream;
    if (p->opts.dtype == GPWENO_F32)
        halo_pack_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(state), static_cast<float *>(send_lo),
                                                        static_cast<float *>(send_hi), layer, G, n, p->dims.ndim + 2,
                                                        p->ncell);
    else
        halo_pack_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(state),
                                                         static_cast<double *>(send_lo), static_cast<double *>(send_hi),
                                                         layer, G, n, p->dims.ndim + 2, p->ncell);
    GPW_CHECK(cudaGetLastError(), "halo pack kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

gpweno_status gpweno_rk3_stage(gpweno_plan p, int stage, void *U, void *scratch, double dt, void *dt_dev,
                               void *stream)
{
    TraceRange tr(stage_range_name(stage));
    g_launches = 0;
    if (!p || p->is_batch || !U || !scratch || stage < 0 || stage > 2) {
        set_error("gpweno_rk3_stage: invalid argument");
        return GPWENO_ERR_ARG;
    }
    if (!aligned16(U) || !aligned16(scratch)) {
        set_error("gpweno_rk3_stage: buffers must be 16-byte aligned");
        return GPWENO_ERR_ARG;
    }
    if (!dt_dev && !(dt > 0.0)) {
        set_error("gpweno_rk3_stage: dt=%g must be positive", dt);
        return GPWENO_ERR_ARG;
    }
    gpweno_status s = check_halo(p, "gpweno_rk3_stage");
    if (s != GPWENO_OK) return s;
    const size_t esz = p->opts.dtype == GPWENO_F32 ? 4 : 8;
    const size_t bytes = esz * (size_t)(p->dims.ndim + 2) * (size_t)p->ncell;
    char *base = static_cast<char *>(scratch);
    const bool cfl = dt_dev && p->opts.cfl > 0.0;
    return launch_stage(p,
                        stage_io(stage, U, base, base + bytes, base + 2 * bytes, base + 3 * bytes, dt,
                                 static_cast<const double *>(dt_dev), cfl),
                        (cudaStream_t)stream);
}

gpweno_status gpweno_rates(gpweno_plan p, const void *U, void *stream)
{
    g_launches = 0;
    if (!p || p->is_batch || !U) {
        set_error("gpweno_rates: invalid argument");
        return GPWENO_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return p->opts.dtype == GPWENO_F32 ? launch_max_rate_f32(p, U, st) : launch_max_rate_f64(p, U, st);
}

gpweno_status gpweno_rate_export(gpweno_plan p, void *rates, void *stream)
{
    g_launches = 0;
    if (!p || !rates) {
        set_error("gpweno_rate_export: invalid argument");
        return GPWENO_ERR_ARG;
    }
    rate_export_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(p->ws, static_cast<unsigned long long *>(rates));
    GPW_CHECK(cudaGetLastError(), "rate export kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

gpweno_status gpweno_dt_from_rates(gpweno_plan p, const void *rates, double cfl, void *dt_dev, void *stream)
{
    g_launches = 0;
    if (!p || !rates || !dt_dev || !(cfl > 0.0)) {
        set_error("gpweno_dt_from_rates: invalid argument");
        return GPWENO_ERR_ARG;
    }
    dt_from_rates_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(static_cast<const unsigned long long *>(rates),
                                                             p->dims.ndim, cfl, static_cast<double *>(dt_dev));
    GPW_CHECK(cudaGetLastError(), "dt kernel launch");
    count_launch(1);
    return GPWENO_OK;
}

gpweno_status gpweno_rk3_step(gpweno_plan p, void *U, void *scratch, double dt, void *dt_dev, void *stream)
{
    TraceRange tr("gpweno_rk3_step");
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
    if (has_external_side(p)) {
        set_error("gpweno_rk3_step: the plan has external sides; step it with gpweno_rk3_stage and a halo "
                  "exchange before each stage");
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
    TraceRange tr("gpweno_cfl_dt");
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
        if (has_external_side(p)) {
            set_error("gpweno_plan_batch: plan %d has external (halo) sides, which batches do not support", k);
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
    TraceRange tr("gpweno_batch_rk3_step");
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
        TraceRange trs(stage_range_name(stage));
        gpweno_status s = b->opts.dtype == GPWENO_F32 ? launch_batch_stage_f32(b, stage, U, scratch, dt, st)
                                                      : launch_batch_stage_f64(b, stage, U, scratch, dt, st);
        if (s != GPWENO_OK) return s;
    }
    return GPWENO_OK;
}

int gpweno_plan_schedule(gpweno_plan p, int *strip_width, int *strips, int *grid, int *ctas_per_sm)
{
    if (!p || p->is_batch || p->dims.ndim != 2) return GPWENO_ERR_ARG;
    if (strip_width) *strip_width = p->sched.W;
    if (strips) *strips = p->sched.nstrips;
    if (grid) *grid = p->sched.grid;
    if (ctas_per_sm) *ctas_per_sm = p->sched.ctas_per_sm;
    return GPWENO_OK;
}

int gpweno_batch_tiles(gpweno_plan b, int *strip_width_cap, int *min_rows, int *ctas_per_slot)
{
    if (!b || !b->is_batch) return GPWENO_ERR_ARG;
    if (strip_width_cap) *strip_width_cap = b->batch_wcap;
    if (min_rows) *min_rows = b->batch_min_rows;
    if (ctas_per_slot) *ctas_per_slot = b->batch_oversub;
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
