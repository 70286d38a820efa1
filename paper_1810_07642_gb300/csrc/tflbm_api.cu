// C-ABI of the thin-film D2Q9 lattice Boltzmann library (include/tflbm.h).
// Owns the population ping-pong buffers, the kappa field and the reduction
// scratch; launches the fused step kernel once per time step, optionally
// replaying a captured CUDA graph of an even number of steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "../../include/tflbm.h"
#include "tflbm_handle.h"

using namespace tflbm;

namespace {

thread_local std::string g_init_err;

int fail(tf_lbm_handle* H, int code, const std::string& msg)
{
    if (H) H->err = msg;
    else g_init_err = msg;
    return code;
}

int cuda_fail(tf_lbm_handle* H, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(H, e == cudaErrorMemoryAllocation ? TF_LBM_ERR_NOMEM : TF_LBM_ERR_CUDA, m);
}

#define CK(H, call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(H, e_, what); \
    } while (0)

// Device pointers only: host memory handed to a kernel would fault or read
// the wrong memory.
int check_dev_ptr(tf_lbm_handle* H, const void* ptr, const char* name, bool allow_null)
{
    if (!ptr) {
        if (allow_null) return TF_LBM_OK;
        return fail(H, TF_LBM_ERR_ARG, std::string(name) + " must not be NULL");
    }
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(H, TF_LBM_ERR_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(H, TF_LBM_ERR_ARG, std::string(name) + " must be device or managed memory");
    int dev = 0;
    cudaGetDevice(&dev);
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(H, TF_LBM_ERR_ARG, std::string(name) + " lives on another device");
    return TF_LBM_OK;
}

void drop_graphs(tf_lbm_handle* H)
{
    for (auto& e : H->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

int validate(const tf_lbm_params* p)
{
    char buf[256];
    auto bad = [&](const char* m) {
        snprintf(buf, sizeof buf, "invalid parameter: %s", m);
        g_init_err = buf;
        return TF_LBM_ERR_ARG;
    };
    if (!p) return bad("params is NULL");
    if (p->nx < 1 || p->ny < 1) return bad("nx and ny must be >= 1");
    if (p->ny > 65535) return bad("ny must be <= 65535");
    if ((long long)p->nx * p->ny > (1LL << 31)) return bad("nx * ny must be <= 2^31");
    if (p->dtype != TF_LBM_F32 && p->dtype != TF_LBM_F64 && p->dtype != TF_LBM_F16 && p->dtype != TF_LBM_BF16)
        return bad("dtype must be TF_LBM_F32, TF_LBM_F64, TF_LBM_F16 or TF_LBM_BF16");
    if (!(p->tau > 0.5)) return bad("tau must be > 1/2");
    if (!(p->hstar > 0.0)) return bad("hstar must be > 0");
    if (!(p->delta >= 0.0)) return bad("delta must be >= 0");
    if (p->n_exp < 1 || p->m_exp < 1 || p->n_exp > 64 || p->m_exp > 64) return bad("n_exp and m_exp must be in [1, 64]");
    if (p->n_exp == p->m_exp) return bad("n_exp must differ from m_exp");
    if (p->pi_sign != 1 && p->pi_sign != -1) return bad("pi_sign must be +1 or -1");
    if (p->forcing != 0 && p->forcing != 1) return bad("forcing must be 0 or 1");
    if (!isfinite(p->gamma) || !isfinite(p->g) || !isfinite(p->gx_body) || !isfinite(p->gy_body) ||
        !isfinite(p->theta_uniform) || !isfinite(p->tau))
        return bad("non-finite parameter");
    return TF_LBM_OK;
}

int store_of(int dtype)
{
    switch (dtype) {
        case TF_LBM_F64: return kStoreF64;
        case TF_LBM_F16: return kStoreF16;
        case TF_LBM_BF16: return kStoreBF16;
        default: return kStoreF32;
    }
}

// Default launch shape: the two-column kernel at tau = 1 where it applies
// (CTAs 64 columns wide for 16-bit storage, 128 for FP32), else the one-column kernel
// with CTAs 128 columns wide (64 on lattices narrower than 1024), and
// a band height that makes the grid one full wave of
// resident CTAs (all bands do the same work, so a partial second wave would
// idle most SMs), but no shorter than 16 rows: each band spends 5 warm-up rows.
Shape default_shape(const tf_lbm_params& p, const Geom& G, bool kfield)
{
    Shape s;
    // two columns per thread at tau = 1 where pairs fit (nx even): it issues
    // fewer instructions per node than the one-column kernel, which is issue
    // bound; 16-bit storage uses it at 64 columns per CTA (one warp), FP32 at
    // 128.  At tau != 1 the one-column kernel is faster in every storage type
    // (the two-column kernel's pulled-population ring costs resident warps)
    const int store = store_of(p.dtype);
    const bool om1 = p.tau == 1.0;
    const bool narrow = store == kStoreF16 || store == kStoreBF16;
    const bool pair = pair_pipeline_ok(G.nx, store) && om1;
    s.block_x = pair ? (narrow ? 64 : 128) : (G.nx >= 1024 ? 128 : 64);
    const int strips = (G.nx + s.block_x - 5) / (s.block_x - 4);  // CTAs overlap by 4 columns
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // otherwise per-thread loads: measured faster than the bulk-copy pipeline
    // on GB300 once loads are prefetched a row ahead
    s.pipeline = pair ? kPipePair : kPipeLdg;
    int occ = step_blocks_per_sm(store_of(p.dtype), s.pipeline, s.block_x, om1, kfield);
    if (occ < 1) occ = 4;
    // bands of balanced height (the kernels spread ny rows over them), as
    // many as fill the resident slots once, but none shorter than 16 rows
    int bands = occ * sms / strips;
    if (bands > G.ny / 16) bands = G.ny / 16;
    if (bands < 1) bands = 1;
    if (bands > 65535) bands = 65535;
    s.bands = bands;
    s.rows = (G.ny + bands - 1) / bands;
    return s;
}

}  // namespace

namespace tflbm {
// Message for tf_lbm_last_error(NULL) from entry points without a handle.
void set_thread_error(const std::string& msg) { g_init_err = msg; }

int handle_fail(tf_lbm_handle* H, int code, const std::string& msg) { return fail(H, code, msg); }
int handle_check_dev_ptr(tf_lbm_handle* H, const void* ptr, const char* name, bool allow_null)
{
    return check_dev_ptr(H, ptr, name, allow_null);
}
void handle_drop_graphs(tf_lbm_handle* H) { drop_graphs(H); }
int sm_count()
{
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}
int handle_cuda_fail(tf_lbm_handle* H, cudaError_t e, const char* what) { return cuda_fail(H, e, what); }

template <typename T>
Consts<T> make_consts(const tf_lbm_handle* H)
{
    Consts<T> C;
    C.gamma = T(H->p.gamma);
    C.g = T(H->p.g);
    C.delta = T(H->p.delta);
    C.hstar = T(H->p.hstar);
    C.nu6 = T(6.0 * (H->p.tau - 0.5) / 3.0);
    C.omega = T(1.0 / H->p.tau);
    C.gx = T(H->p.gx_body);
    C.gy = T(H->p.gy_body);
    C.kappa_u = T(H->kappa_u);
    C.pi_sgn = T(H->p.pi_sign);
    C.href = T(H->href);
    C.mscale = T(H->desc.mscale);
    C.minv = T(H->desc.minv);
    C.r_axis = T(H->desc.r_axis);
    C.r_diag = T(H->desc.r_diag);
    C.nr_axis = T(-H->desc.r_axis * H->desc.mscale);
    C.nr_diag = T(-H->desc.r_diag * H->desc.mscale);
    C.r_sum = T(4.0 * (H->desc.r_axis + H->desc.r_diag));
    C.n_exp = H->p.n_exp;
    C.m_exp = H->p.m_exp;
    C.status = H->status;
    C.wait_limit = H->wait_limit;
    C.forcing = H->p.forcing;
    C.flip = 0;
    return C;
}

cudaError_t launch_one_step(tf_lbm_handle* H, int from, cudaStream_t st)
{
    Consts<float> c32 = make_consts<float>(H);
    Consts<double> c64 = make_consts<double>(H);
    c32.flip = c64.flip = from & 1;
    return launch_step(H->desc.store, H->buf[from], H->buf[from ^ 1], H->kappa, H->G, &c32, &c64,
                       H->shape, st);
}

cudaError_t launch_step_between(tf_lbm_handle* H, const void* fin, void* fout, cudaStream_t st)
{
    const Consts<float> c32 = make_consts<float>(H);
    const Consts<double> c64 = make_consts<double>(H);
    return launch_step(H->desc.store, fin, fout, H->kappa, H->G, &c32, &c64, H->shape, st);
}

template Consts<float> make_consts<float>(const tf_lbm_handle*);
template Consts<double> make_consts<double>(const tf_lbm_handle*);
}  // namespace tflbm

static_assert(kStatusTimeout == TF_LBM_STATUS_TIMEOUT, "status bits out of sync");

extern "C" {

int32_t tf_lbm_version(void) { return 200; }

const char* tf_lbm_last_error(const tf_lbm_handle* H)
{
    return H ? H->err.c_str() : g_init_err.c_str();
}

int tf_lbm_init(tf_lbm_handle** out, const tf_lbm_params* params, const void* h0,
                const void* theta, void* stream)
{
    g_init_err.clear();
    if (!out) return fail(nullptr, TF_LBM_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    int rc = validate(params);
    if (rc) return rc;
    if ((rc = check_dev_ptr(nullptr, h0, "h0", false))) return rc;
    if ((rc = check_dev_ptr(nullptr, theta, "theta", true))) return rc;

    tf_lbm_handle* H = new tf_lbm_handle();
    H->p = *params;
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetDevice(&H->device);
    H->desc.store = store_of(params->dtype);
    H->dbl = params->dtype == TF_LBM_F64;
    H->esize = H->dbl ? 8 : 4;
    H->msize = (params->dtype == TF_LBM_F16 || params->dtype == TF_LBM_BF16) ? 2 : H->esize;
    const int align = 128 / (int)H->msize;  // rows of every plane start on 128-byte boundaries
    H->G.nx = params->nx;
    H->G.ny = params->ny;
    H->G.pitch = (params->nx + align - 1) / align * align;
    H->G.plane = (long long)params->ny * H->G.pitch;
    if (9LL * H->G.plane >= (1LL << 31)) {  // the step kernel uses 32-bit element offsets
        delete H;
        return fail(nullptr, TF_LBM_ERR_UNSUPPORTED,
                    "lattice too large: 9 * ny * pitch must stay below 2^31 elements");
    }
    H->shape = default_shape(*params, H->G, theta != nullptr);
    H->graph_chunk = ((long long)params->nx * params->ny <= (1LL << 20)) ? 64 : 0;

    auto bail = [&](int code) {
        g_init_err = H->err;
        tf_lbm_destroy(H);
        return code;
    };
    const size_t bytes = (size_t)H->G.plane * (H->esize + 8 * H->msize);
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&H->buf[b], bytes)) != cudaSuccess) return bail(cuda_fail(H, e, "cudaMalloc populations"));
        if ((e = cudaMemsetAsync(H->buf[b], 0, bytes, st)) != cudaSuccess) return bail(cuda_fail(H, e, "cudaMemsetAsync"));
    }
    H->nmass = mass_blocks(H->G);
    if (H->nmass < kSumBlocks) H->nmass = kSumBlocks;
    if ((e = cudaMalloc(&H->partials, sizeof(double) * 2 * H->nmass + sizeof(double))) != cudaSuccess)
        return bail(cuda_fail(H, e, "cudaMalloc scratch"));
    H->result = H->partials + 2 * H->nmass;
    if ((e = cudaMalloc(&H->flag, 2 * sizeof(int))) != cudaSuccess) return bail(cuda_fail(H, e, "cudaMalloc flag"));
    H->status = H->flag + 1;
    if ((e = cudaMemsetAsync(H->flag, 0, 2 * sizeof(int), st)) != cudaSuccess) return bail(cuda_fail(H, e, "cudaMemsetAsync"));

    const double kscale = (double)(params->n_exp - 1) * (params->m_exp - 1) /
                          ((double)(params->n_exp - params->m_exp) * params->hstar);
    const long long n = (long long)params->nx * params->ny;
    if (theta) {
        if ((e = cudaMalloc(&H->kappa, n * H->esize)) != cudaSuccess) return bail(cuda_fail(H, e, "cudaMalloc kappa"));
        e = aux_kappa(H->dbl, H->kappa, theta, params->nx, params->ny, params->n_exp, params->m_exp,
                      params->hstar, st);
        if (e != cudaSuccess) return bail(cuda_fail(H, e, "kappa kernel"));
    } else {
        H->kappa_u = (1.0 - cos(params->theta_uniform)) * kscale;
    }
    // Reference height: the smallest h0, rounded to the storage type.  Plane
    // 0 stores f_0 - href, so FP32 resolves h - href to 2^-24 of |h - href|:
    // the thin parts of a film (precursor, contact lines), where the
    // disjoining pressure is stiffest and rounding differences grow fastest,
    // get the finest resolution, while thick parts keep 2^-24 relative.
    e = aux_min(H->dbl, h0, n, H->partials, H->nmass, H->result, st);
    if (e != cudaSuccess) return bail(cuda_fail(H, e, "min kernel"));
    double hmin = 0.0;
    if ((e = cudaMemcpyAsync(&hmin, H->result, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(H, e, "reading the smallest height"));
    H->href = H->dbl ? hmin : (double)(float)hmin;
    if (!isfinite(H->href)) H->href = 0.0;  // a non-finite h0 is reported by tf_lbm_check
    // 16-bit storage of the moving populations: deviations from the rest
    // equilibrium at href, scaled by 2^10 in FP16 (keeps small deviations out
    // of the subnormal range; |f_l| up to 64 stays finite), unscaled in BF16.
    H->desc.href = H->href;
    H->desc.mscale = params->dtype == TF_LBM_F16 ? 1024.0 : 1.0;
    H->desc.minv = 1.0 / H->desc.mscale;
    if (H->msize == 2) {
        H->desc.r_axis = (double)(float)(params->g * H->href * H->href / 6.0);
        H->desc.r_diag = (double)(float)(params->g * H->href * H->href / 24.0);
    }
    e = aux_init(H->desc, H->buf[0], h0, H->G, params->g, st);
    if (e != cudaSuccess) return bail(cuda_fail(H, e, "init kernel"));
    H->cur = 0;
    *out = H;
    return TF_LBM_OK;
}

int tf_lbm_step(tf_lbm_handle* H, int64_t nsteps, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(H, TF_LBM_ERR_ARG, "nsteps must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int chunk = H->graph_chunk;
    while (nsteps > 0) {
        if (chunk > 0 && nsteps >= chunk) {
            cudaGraphExec_t& ex = H->exec[H->cur];
            if (!ex) {
                if (!H->cap) CK(H, cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking), "cudaStreamCreate");
                CK(H, cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
                cudaError_t le = cudaSuccess;
                for (int i = 0; i < chunk && le == cudaSuccess; ++i) le = launch_one_step(H, H->cur ^ (i & 1), H->cap);
                cudaGraph_t g = nullptr;
                cudaError_t ce = cudaStreamEndCapture(H->cap, &g);
                if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(H, le, "step kernel (capture)"); }
                if (ce != cudaSuccess) return cuda_fail(H, ce, "cudaStreamEndCapture");
                cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) { ex = nullptr; return cuda_fail(H, ie, "cudaGraphInstantiate"); }
            }
            CK(H, cudaGraphLaunch(ex, st), "cudaGraphLaunch");
            nsteps -= chunk;
            H->time += chunk;
        } else {
            CK(H, launch_one_step(H, H->cur, st), "step kernel");
            H->cur ^= 1;
            --nsteps;
            ++H->time;
        }
    }
    return TF_LBM_OK;
}

int tf_lbm_moments(tf_lbm_handle* H, void* h, void* ux, void* uy, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    int rc;
    if ((rc = check_dev_ptr(H, h, "h", true)) || (rc = check_dev_ptr(H, ux, "ux", true)) ||
        (rc = check_dev_ptr(H, uy, "uy", true)))
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = aux_moments(H->desc, H->buf[H->cur], h, ux, uy, H->G, st);
    CK(H, e, "moments kernel");
    return TF_LBM_OK;
}

int tf_lbm_pressure_force(tf_lbm_handle* H, void* p, void* fx, void* fy, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    int rc;
    if ((rc = check_dev_ptr(H, p, "p", true)) || (rc = check_dev_ptr(H, fx, "fx", true)) ||
        (rc = check_dev_ptr(H, fy, "fy", true)))
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)H->G.nx * H->G.ny;
    if (!H->diag) CK(H, cudaMalloc(&H->diag, 2 * n * H->esize), "cudaMalloc diagnostics");
    const Consts<float> c32 = make_consts<float>(H);
    const Consts<double> c64 = make_consts<double>(H);
    char* sc = (char*)H->diag;
    cudaError_t e = aux_pressure_force(H->desc, H->buf[H->cur], H->kappa, p, fx, fy, sc, sc + n * H->esize,
                                       H->G, &c32, &c64, st);
    CK(H, e, "pressure/force kernels");
    return TF_LBM_OK;
}

int tf_lbm_mass(tf_lbm_handle* H, double* mass_host, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (!mass_host) return fail(H, TF_LBM_ERR_ARG, "mass_host must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = aux_mass(H->desc, H->buf[H->cur], H->G, H->partials, H->nmass, H->result, st);
    CK(H, e, "mass kernels");
    CK(H, cudaMemcpyAsync(mass_host, H->result, sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(H, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    // plane 0 stores f_0 - href: add href back once per node
    *mass_host += H->href * (double)H->G.nx * (double)H->G.ny;
    return TF_LBM_OK;
}

int tf_lbm_check(tf_lbm_handle* H, int32_t* status_host, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (!status_host) return fail(H, TF_LBM_ERR_ARG, "status_host must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    CK(H, cudaMemsetAsync(H->flag, 0, sizeof(int), st), "cudaMemsetAsync");
    cudaError_t e = aux_check(H->desc, H->buf[H->cur], H->G, H->flag, st);
    CK(H, e, "check kernel");
    int v[2] = {0, 0};
    CK(H, cudaMemcpyAsync(v, H->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(H, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *status_host = v[0] | v[1];
    return TF_LBM_OK;
}

int tf_lbm_get_state(tf_lbm_handle* H, void* f, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    int rc;
    if ((rc = check_dev_ptr(H, f, "f", false))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = aux_get_state(H->desc, H->buf[H->cur], (double*)f, H->G, st);
    CK(H, e, "get_state kernel");
    return TF_LBM_OK;
}

int tf_lbm_set_state(tf_lbm_handle* H, const void* f, void* stream)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    int rc;
    if ((rc = check_dev_ptr(H, f, "f", false))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = aux_set_state(H->desc, H->buf[H->cur], (const double*)f, H->G, st);
    CK(H, e, "set_state kernel");
    return TF_LBM_OK;
}

int64_t tf_lbm_time(const tf_lbm_handle* H) { return H ? H->time : -1; }

int tf_lbm_get_launch(const tf_lbm_handle* H, tf_lbm_launch* out)
{
    if (!H || !out) return TF_LBM_ERR_ARG;
    out->block_x = H->shape.block_x;
    out->rows = H->shape.rows;
    out->graph_chunk = H->graph_chunk;
    out->pipeline = H->shape.pipeline;
    return TF_LBM_OK;
}

int tf_lbm_set_launch(tf_lbm_handle* H, const tf_lbm_launch* in)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (!in) return fail(H, TF_LBM_ERR_ARG, "launch is NULL");
    const int bx = in->block_x;
    if (bx != 64 && bx != 128 && bx != 256) return fail(H, TF_LBM_ERR_ARG, "block_x must be 64, 128 or 256");
    if (in->rows < 1 || in->rows > 65535) return fail(H, TF_LBM_ERR_ARG, "rows must be in [1, 65535]");
    if (in->graph_chunk < 0 || (in->graph_chunk % 2) != 0 || in->graph_chunk > 4096)
        return fail(H, TF_LBM_ERR_ARG, "graph_chunk must be 0 or an even number <= 4096");
    if (in->pipeline != kPipeTma && in->pipeline != kPipeLdg && in->pipeline != kPipeAsync &&
        in->pipeline != kPipePair)
        return fail(H, TF_LBM_ERR_ARG,
                    "pipeline must be 0 (bulk copies), 1 (per-thread loads), 2 (per-thread async copies) "
                    "or 3 (two columns per thread)");
    if (in->pipeline == kPipePair && !pair_pipeline_ok(H->G.nx, H->desc.store))
        return fail(H, TF_LBM_ERR_ARG, "the two-column pipeline needs nx even and an FP32 compute type");
    if (in->pipeline == kPipeAsync && H->msize != H->esize)
        return fail(H, TF_LBM_ERR_ARG, "the async-copy pipeline needs FP32 or FP64 storage");
    if (in->pipeline == kPipeTma && !tma_pipeline_ok(H->G.nx))
        return fail(H, TF_LBM_ERR_ARG, "the bulk-copy pipeline needs nx to be a multiple of 8 and >= 16");
    drop_graphs(H);
    H->shape.pipeline = in->pipeline;
    H->shape.block_x = bx;
    H->shape.rows = in->rows;
    H->shape.bands = 0;
    H->graph_chunk = in->graph_chunk;
    return TF_LBM_OK;
}

int tf_lbm_set_wait_limit(tf_lbm_handle* H, int32_t polls)
{
    if (!H) return fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    H->wait_limit = polls < 0 ? kWaitLimit : polls;
    drop_graphs(H);  // captured launches carry the old limit
    return TF_LBM_OK;
}

void tf_lbm_destroy(tf_lbm_handle* H)
{
    if (!H) return;
    cudaDeviceSynchronize();
    drop_graphs(H);
    if (H->cap) cudaStreamDestroy(H->cap);
    for (auto& b : H->buf)
        if (b) cudaFree(b);
    if (H->kappa) cudaFree(H->kappa);
    if (H->partials) cudaFree(H->partials);
    if (H->flag) cudaFree(H->flag);
    if (H->diag) cudaFree(H->diag);
    if (H->adj) cudaFree(H->adj);
    if (H->dscr) cudaFree(H->dscr);
    if (H->tscr) cudaFree(H->tscr);
    delete H;
}

}  // extern "C"
