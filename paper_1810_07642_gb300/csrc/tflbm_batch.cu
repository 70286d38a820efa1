// Batches of independent simulations (parameter sweeps over uneven domains),
// the launch-shape autotuner and the on-device film diagnostics
// (include/tflbm.h).
//
// A batched step is one launch of k_step_batch (one column per thread) or
// k_step2_batch (two columns per thread, every nx even, FP32 compute type)
// over a flat table of work items (domain, column strip, row band); a table
// of per-domain records
// (geometry, constants, the two population buffers, kappa) lives in device
// memory next to it.  The records name the buffers in the order they had
// when the table was written; a phase bit counts the steps since then, so a
// captured CUDA graph of an even number of steps stays valid for the whole
// run.  Per-handle calls in between (tf_lbm_step on one handle) are detected
// from the handles' own buffer indices and the table is rewritten.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tflbm.h"
#include "tflbm_handle.h"

using namespace tflbm;

namespace tflbm {
void set_thread_error(const std::string& msg);  // defined in tflbm_api.cu
}

struct tf_lbm_batch {
    std::vector<tf_lbm_handle*> hs;
    int store = kStoreF32;
    bool dbl = false;
    bool om1 = false;  // every domain has omega == 1 in the compute type
    bool kf = false;   // some domain has a kappa field: every domain gets one
    bool pair_ok = false;  // the two-column kernel applies (FP32 compute type, every nx even)
    std::vector<void*> kfill;  // filled kappa fields of the uniform domains (kf only)
    std::vector<int> cur0;     // each handle's buffer index when the table was written
    int phase = 0;             // steps taken since then, mod 2
    void* doms = nullptr;      // BatchDomain<compute type>[count]
    BatchItem* items = nullptr;
    int item_cap = 0;
    int nitems = 0;
    int* queue = nullptr;  // item counter and finished-CTA counter (zero between launches)
    int grid = 0;
    tf_lbm_batch_launch L{64, 64, 0, 0, kPipeLdg};
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    double* dpart = nullptr;  // diagnostics partials
    std::string err;
};

namespace {

constexpr int kDiagBlocksPerDomain = 64;

int bfail(tf_lbm_batch* B, int code, const std::string& msg)
{
    if (B) B->err = msg;
    else set_thread_error(msg);
    return code;
}

int bcuda(tf_lbm_batch* B, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return bfail(B, e == cudaErrorMemoryAllocation ? TF_LBM_ERR_NOMEM : TF_LBM_ERR_CUDA, m);
}

#define BCK(B, call, what)                                 \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(B, e_, what);  \
    } while (0)

template <typename T>
__global__ void k_fill(T* p, long long n, T v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

template <typename T>
BatchDomain<T> domain_of(const tf_lbm_handle* H, int from, const void* kappa)
{
    BatchDomain<T> D;
    D.G = H->G;
    D.C = make_consts<T>(H);
    D.buf[0] = H->buf[from];
    D.buf[1] = H->buf[from ^ 1];
    D.kappa = (const T*)kappa;
    return D;
}

size_t domain_bytes(bool dbl) { return dbl ? sizeof(BatchDomain<double>) : sizeof(BatchDomain<float>); }

void drop_batch_graphs(tf_lbm_batch* B)
{
    for (auto& e : B->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

int strips_of(int nx, int bx) { return (nx + bx - 5) / (bx - 4); }  // CTAs overlap by 4 columns
int bands_of(int ny, int rows) { return (ny + rows - 1) / rows; }

long long count_items(const tf_lbm_batch* B, int bx, int rows)
{
    long long n = 0;
    for (auto* H : B->hs) n += (long long)strips_of(H->G.nx, bx) * bands_of(H->G.ny, rows);
    return n;
}

// Smallest band height (>= 16, <= the tallest domain) whose items fit in
// `slots` CTAs.
int rows_for_slots(const tf_lbm_batch* B, int bx, long long slots)
{
    int ymax = 1;
    for (auto* H : B->hs) ymax = std::max(ymax, H->G.ny);
    int lo = std::min(16, ymax), hi = ymax;
    if (count_items(B, bx, lo) <= slots) return lo;
    while (hi - lo > 1) {  // count_items decreases as rows grows
        const int mid = (lo + hi) / 2;
        if (count_items(B, bx, mid) <= slots) hi = mid;
        else lo = mid;
    }
    return hi;
}

int batch_occupancy(const tf_lbm_batch* B, int bx, int pipeline)
{
    int occ = 0;
    BatchLaunch q{};
    q.block_x = bx;
    q.pair = pipeline == kPipePair;
    q.omega1 = B->om1;
    q.kfield = B->kf;
    q.query_occupancy = &occ;
    if (launch_step_batch(B->store, q, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ;
}

// Write the per-domain table for the handles' current buffer indices.
int write_table(tf_lbm_batch* B, cudaStream_t st)
{
    const int n = (int)B->hs.size();
    std::vector<char> host(domain_bytes(B->dbl) * n);
    for (int d = 0; d < n; ++d) {
        tf_lbm_handle* H = B->hs[d];
        const void* kap = B->kf ? (H->kappa ? H->kappa : B->kfill[d]) : nullptr;
        if (B->dbl) ((BatchDomain<double>*)host.data())[d] = domain_of<double>(H, H->cur, kap);
        else ((BatchDomain<float>*)host.data())[d] = domain_of<float>(H, H->cur, kap);
        B->cur0[d] = H->cur;
    }
    B->phase = 0;
    // pageable source: the call returns once `host` has been staged
    BCK(B, cudaMemcpyAsync(B->doms, host.data(), host.size(), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync table");
    return TF_LBM_OK;
}

// Rewrite the table if some handle was stepped on its own since it was
// written (its buffer index no longer follows the batch's phase).
int sync_table(tf_lbm_batch* B, cudaStream_t st)
{
    for (size_t d = 0; d < B->hs.size(); ++d)
        if (B->hs[d]->cur != (B->cur0[d] ^ B->phase)) return write_table(B, st);
    return TF_LBM_OK;
}

// Build the work items of a launch shape: domains in order, bands of a
// domain in order, strips fastest (as the single-domain grid orders them).
int write_items(tf_lbm_batch* B, const tf_lbm_batch_launch& L, cudaStream_t st)
{
    const long long n = count_items(B, L.block_x, L.rows);
    if (n > (1LL << 30)) return bfail(B, TF_LBM_ERR_ARG, "too many work items: raise rows");
    std::vector<BatchItem> host;
    host.reserve((size_t)n);
    for (int d = 0; d < (int)B->hs.size(); ++d) {
        const Geom& G = B->hs[d]->G;
        const int ns = strips_of(G.nx, L.block_x), nb = bands_of(G.ny, L.rows);
        for (int b = 0; b < nb; ++b)
            for (int s = 0; s < ns; ++s) host.push_back(BatchItem{d, s, b, nb});
    }
    if ((int)n > B->item_cap) {
        if (B->items) cudaFree(B->items);
        B->items = nullptr;
        B->item_cap = 0;
        BCK(B, cudaMalloc(&B->items, n * sizeof(BatchItem)), "cudaMalloc items");
        B->item_cap = (int)n;
    }
    BCK(B, cudaMemcpyAsync(B->items, host.data(), n * sizeof(BatchItem), cudaMemcpyHostToDevice, st),
        "cudaMemcpyAsync items");
    B->nitems = (int)n;
    int grid = (int)n;
    if (L.queue) {
        const int occ = batch_occupancy(B, L.block_x, L.pipeline);
        const long long slots = (long long)std::max(occ, 1) * sm_count();
        grid = (int)std::min<long long>(n, slots);
    }
    B->grid = grid;
    return TF_LBM_OK;
}

cudaError_t launch_batch(tf_lbm_batch* B, int parity, cudaStream_t st)
{
    BatchLaunch q{};
    q.block_x = B->L.block_x;
    q.pair = B->L.pipeline == kPipePair;
    q.omega1 = B->om1;
    q.kfield = B->kf;
    q.items = B->items;
    q.nitems = B->nitems;
    q.doms = B->doms;
    q.parity = parity;
    q.queue = B->L.queue ? B->queue : nullptr;
    q.grid = B->grid;
    return launch_step_batch(B->store, q, st);
}

int validate_batch_launch(tf_lbm_batch* B, const tf_lbm_batch_launch* in)
{
    if (!in) return bfail(B, TF_LBM_ERR_ARG, "launch is NULL");
    if (in->block_x != 64 && in->block_x != 128 && in->block_x != 256)
        return bfail(B, TF_LBM_ERR_ARG, "block_x must be 64, 128 or 256");
    if (in->rows < 1 || in->rows > 65535) return bfail(B, TF_LBM_ERR_ARG, "rows must be in [1, 65535]");
    if (in->graph_chunk < 0 || (in->graph_chunk % 2) != 0 || in->graph_chunk > 4096)
        return bfail(B, TF_LBM_ERR_ARG, "graph_chunk must be 0 or an even number <= 4096");
    if (in->queue != 0 && in->queue != 1) return bfail(B, TF_LBM_ERR_ARG, "queue must be 0 or 1");
    if (in->pipeline != kPipeLdg && in->pipeline != kPipePair)
        return bfail(B, TF_LBM_ERR_ARG, "pipeline must be 1 (one column per thread) or 3 (two columns per thread)");
    if (in->pipeline == kPipePair && !B->pair_ok)
        return bfail(B, TF_LBM_ERR_ARG, "the two-column pipeline needs every nx even and an FP32 compute type");
    return TF_LBM_OK;
}

int apply_launch(tf_lbm_batch* B, const tf_lbm_batch_launch& L, cudaStream_t st)
{
    drop_batch_graphs(B);
    const tf_lbm_batch_launch old = B->L;
    B->L = L;
    int rc = write_items(B, L, st);
    if (rc) B->L = old;
    return rc;
}

// Time `steps` (even) launches of the current shape, after two untimed ones.
int time_batch(tf_lbm_batch* B, int steps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    int parity = B->phase;
    for (int i = 0; i < 2; ++i, parity ^= 1) BCK(B, launch_batch(B, parity, st), "batched step (tuning)");
    BCK(B, cudaEventRecord(e0, st), "cudaEventRecord");
    for (int i = 0; i < steps; ++i, parity ^= 1) BCK(B, launch_batch(B, parity, st), "batched step (tuning)");
    BCK(B, cudaEventRecord(e1, st), "cudaEventRecord");
    BCK(B, cudaEventSynchronize(e1), "cudaEventSynchronize");
    BCK(B, cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
    return TF_LBM_OK;
}

// Time candidates (first pass over all, second over the four fastest) and
// return the index of the fastest.
template <typename Cand, typename TimeFn>
int pick_fastest(const std::vector<Cand>& cands, TimeFn time_one, int* rc)
{
    std::vector<std::pair<float, int>> t;
    for (int i = 0; i < (int)cands.size(); ++i) {
        float ms = 0.f;
        if ((*rc = time_one(cands[i], &ms))) return -1;
        t.push_back({ms, i});
    }
    std::sort(t.begin(), t.end());
    const int top = std::min<int>(4, (int)t.size());
    for (int k = 0; k < top; ++k) {
        float ms = 0.f;
        if ((*rc = time_one(cands[t[k].second], &ms))) return -1;
        t[k].first = std::min(t[k].first, ms);
    }
    std::sort(t.begin(), t.begin() + top);
    return t.empty() ? -1 : t[0].second;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------- single handle

int tf_lbm_tune(tf_lbm_handle* H, int32_t trial_steps, tf_lbm_launch* best, void* stream)
{
    if (!H) {
        set_thread_error("handle is NULL");
        return TF_LBM_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int steps = trial_steps <= 0 ? 16 : (trial_steps + 1) / 2 * 2;
    const bool kf = H->kappa != nullptr;
    const bool om1 = H->dbl ? make_consts<double>(H).omega == 1.0 : make_consts<float>(H).omega == 1.0f;
    const int sms = sm_count();

    // candidate shapes
    std::vector<Shape> cands;
    for (int bx : {64, 128, 256}) {
        const int strips = strips_of(H->G.nx, bx);
        for (int pipe : {kPipePair, kPipeLdg, kPipeAsync, kPipeTma}) {
            if (pipe == kPipeTma && !tma_pipeline_ok(H->G.nx)) continue;
            if (pipe == kPipeAsync && H->msize != H->esize) continue;
            if (pipe == kPipePair && !pair_pipeline_ok(H->G.nx, H->desc.store)) continue;
            const int occ = std::max(1, step_blocks_per_sm(H->desc.store, pipe, bx, om1, kf));
            std::vector<int> rows;
            for (int w = 1; w <= 3; ++w) {
                const int bands = std::max(1, w * occ * sms / strips);
                rows.push_back(std::max(16, (H->G.ny + bands - 1) / bands));
                // balanced bands filling w waves exactly (rows need not divide ny)
                if (bands <= std::min(65535, H->G.ny / 16)) {
                    Shape s;
                    s.block_x = bx;
                    s.pipeline = pipe;
                    s.bands = bands;
                    s.rows = (H->G.ny + bands - 1) / bands;
                    cands.push_back(s);
                }
            }
            for (int r : {2, 4, 8, 16, 32, 64, 128, 256}) rows.push_back(r);
            for (int r : rows) {
                r = std::min(r, std::max(H->G.ny, 1));
                Shape s;
                s.block_x = bx;
                s.rows = r;
                s.pipeline = pipe;
                bool dup = false;
                for (auto& c : cands) dup |= c.block_x == bx && c.rows == r && c.pipeline == pipe && c.bands == 0;
                if (!dup) cands.push_back(s);
            }
        }
    }

    const size_t bytes = (size_t)H->G.plane * (H->esize + 8 * H->msize);
    void* snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, bytes);
    if (e != cudaSuccess) return handle_cuda_fail(H, e, "cudaMalloc tuning snapshot");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TF_LBM_OK;
    const Shape old = H->shape;
    auto finish = [&](int code) {
        // put the state back and release the scratch, whatever happened
        cudaError_t r = cudaMemcpyAsync(H->buf[H->cur], snap, bytes, cudaMemcpyDeviceToDevice, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(snap);
        if (code == TF_LBM_OK && r != cudaSuccess) return handle_cuda_fail(H, r, "restoring the state after tuning");
        return code;
    };
    if ((e = cudaMemcpyAsync(snap, H->buf[H->cur], bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return finish(handle_cuda_fail(H, e, "tuning setup"));

    auto time_one = [&](const Shape& s, float* ms) -> int {
        H->shape = s;
        int from = H->cur;
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < 2 && r == cudaSuccess; ++i, from ^= 1) r = launch_one_step(H, from, st);
        if (r == cudaSuccess) r = cudaEventRecord(e0, st);
        for (int i = 0; i < steps && r == cudaSuccess; ++i, from ^= 1) r = launch_one_step(H, from, st);
        if (r == cudaSuccess) r = cudaEventRecord(e1, st);
        if (r == cudaSuccess) r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        return r == cudaSuccess ? TF_LBM_OK : handle_cuda_fail(H, r, "step kernel (tuning)");
    };
    const int k = pick_fastest(cands, time_one, &rc);
    if (rc) {
        H->shape = old;
        return finish(rc);
    }
    H->shape = cands[k];
    if (H->shape.block_x != old.block_x || H->shape.rows != old.rows || H->shape.pipeline != old.pipeline ||
        H->shape.bands != old.bands)
        handle_drop_graphs(H);
    if (best) {
        best->block_x = H->shape.block_x;
        best->rows = H->shape.rows;
        best->graph_chunk = H->graph_chunk;
        best->pipeline = H->shape.pipeline;
    }
    return finish(TF_LBM_OK);
}

int tf_lbm_diagnostics(tf_lbm_handle* H, double h_wet, int32_t mode_x, int32_t mode_y, void* out, void* stream)
{
    if (!H) {
        set_thread_error("handle is NULL");
        return TF_LBM_ERR_ARG;
    }
    int rc = handle_check_dev_ptr(H, out, "out", false);
    if (rc) return rc;
    if (isnan(h_wet)) return handle_fail(H, TF_LBM_ERR_ARG, "h_wet is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)H->G.nx * H->G.ny;
    const int nb = (int)std::min<long long>(kSumBlocks, std::max<long long>(1, n / (256LL * 16)));
    const size_t tab = 256;  // one BatchDomain record, padded
    static_assert(sizeof(BatchDomain<double>) <= 256, "diagnostics record too large");
    if (!H->dscr) {
        cudaError_t e = cudaMalloc(&H->dscr, tab + sizeof(double) * diag_partials(1, kSumBlocks));
        if (e != cudaSuccess) {
            H->dscr = nullptr;
            return handle_cuda_fail(H, e, "cudaMalloc diagnostics scratch");
        }
    }
    BatchDomain<double> d64;
    BatchDomain<float> d32;
    const void* rec = H->dbl ? (const void*)&d64 : (const void*)&d32;
    if (H->dbl) d64 = domain_of<double>(H, H->cur, H->kappa);
    else d32 = domain_of<float>(H, H->cur, H->kappa);
    cudaError_t e = cudaMemcpyAsync(H->dscr, rec, domain_bytes(H->dbl), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return handle_cuda_fail(H, e, "cudaMemcpyAsync diagnostics record");
    e = aux_diag(H->desc.store, H->dscr, 1, 0, h_wet, mode_x, mode_y, (double*)((char*)H->dscr + tab), nb,
                 (double*)out, st);
    if (e != cudaSuccess) return handle_cuda_fail(H, e, "diagnostics kernels");
    return TF_LBM_OK;
}

int tf_lbm_term_norms(tf_lbm_handle* H, void* out, void* stream)
{
    if (!H) {
        set_thread_error("handle is NULL");
        return TF_LBM_ERR_ARG;
    }
    int rc = handle_check_dev_ptr(H, out, "out", false);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)H->G.nx * H->G.ny;
    const int nb = (int)std::min<long long>(kSumBlocks, std::max<long long>(1, n / (256LL * 16)));
    const size_t fields = (5 * n * H->esize + 255) / 256 * 256;
    if (!H->tscr) {
        cudaError_t e = cudaMalloc(&H->tscr, fields + 6 * sizeof(double) * kSumBlocks);
        if (e != cudaSuccess) {
            H->tscr = nullptr;
            return handle_cuda_fail(H, e, "cudaMalloc term-norm scratch");
        }
    }
    const Consts<float> c32 = make_consts<float>(H);
    const Consts<double> c64 = make_consts<double>(H);
    cudaError_t e = aux_term_norms(H->desc, H->buf[H->cur], H->kappa, H->G, &c32, &c64, H->tscr,
                                   (double*)((char*)H->tscr + fields), nb, (double*)out, st);
    if (e != cudaSuccess) return handle_cuda_fail(H, e, "term-norm kernels");
    return TF_LBM_OK;
}

// -------------------------------------------------------------------- batch

const char* tf_lbm_batch_last_error(const tf_lbm_batch* B)
{
    return B ? B->err.c_str() : tf_lbm_last_error(nullptr);
}

void tf_lbm_batch_destroy(tf_lbm_batch* B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    drop_batch_graphs(B);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (void* p : B->kfill)
        if (p) cudaFree(p);
    if (B->doms) cudaFree(B->doms);
    if (B->items) cudaFree(B->items);
    if (B->queue) cudaFree(B->queue);
    if (B->dpart) cudaFree(B->dpart);
    delete B;
}

int tf_lbm_batch_create(tf_lbm_batch** out, tf_lbm_handle* const* handles, int32_t count, void* stream)
{
    if (!out) return bfail(nullptr, TF_LBM_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    if (!handles || count < 1) return bfail(nullptr, TF_LBM_ERR_ARG, "need count >= 1 handles");
    for (int i = 0; i < count; ++i) {
        if (!handles[i]) return bfail(nullptr, TF_LBM_ERR_ARG, "handle " + std::to_string(i) + " is NULL");
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i])
                return bfail(nullptr, TF_LBM_ERR_ARG, "handle " + std::to_string(i) + " appears twice");
        if (handles[i]->p.dtype != handles[0]->p.dtype)
            return bfail(nullptr, TF_LBM_ERR_ARG, "all handles of a batch must have the same dtype");
    }
    cudaStream_t st = (cudaStream_t)stream;
    tf_lbm_batch* B = new tf_lbm_batch();
    B->hs.assign(handles, handles + count);
    B->store = handles[0]->desc.store;
    B->dbl = handles[0]->dbl;
    B->cur0.assign(count, 0);
    B->kfill.assign(count, nullptr);
    B->om1 = true;
    B->pair_ok = !B->dbl;
    for (auto* H : B->hs) {
        B->kf |= H->kappa != nullptr;
        B->om1 &= B->dbl ? make_consts<double>(H).omega == 1.0 : make_consts<float>(H).omega == 1.0f;
        B->pair_ok &= pair_pipeline_ok(H->G.nx, B->store);
    }
    auto bail = [&](int code) {
        set_thread_error(B->err);
        tf_lbm_batch_destroy(B);
        return code;
    };
    cudaError_t e;
    if (B->kf) {
        for (int d = 0; d < count; ++d) {
            tf_lbm_handle* H = B->hs[d];
            if (H->kappa) continue;
            const long long n = (long long)H->G.nx * H->G.ny;
            if ((e = cudaMalloc(&B->kfill[d], n * H->esize)) != cudaSuccess) return bail(bcuda(B, e, "cudaMalloc kappa"));
            const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
            if (B->dbl) k_fill<double><<<blocks, 256, 0, st>>>((double*)B->kfill[d], n, H->kappa_u);
            else k_fill<float><<<blocks, 256, 0, st>>>((float*)B->kfill[d], n, make_consts<float>(H).kappa_u);
            if ((e = cudaGetLastError()) != cudaSuccess) return bail(bcuda(B, e, "fill kernel"));
        }
    }
    if ((e = cudaMalloc(&B->doms, domain_bytes(B->dbl) * count)) != cudaSuccess)
        return bail(bcuda(B, e, "cudaMalloc domain table"));
    if ((e = cudaMalloc(&B->queue, 2 * sizeof(int))) != cudaSuccess) return bail(bcuda(B, e, "cudaMalloc queue"));
    if ((e = cudaMemsetAsync(B->queue, 0, 2 * sizeof(int), st)) != cudaSuccess) return bail(bcuda(B, e, "cudaMemsetAsync"));
    const size_t dp = diag_partials(count, kDiagBlocksPerDomain);
    if ((e = cudaMalloc(&B->dpart, dp * sizeof(double))) != cudaSuccess) return bail(bcuda(B, e, "cudaMalloc diagnostics"));
    int rc = write_table(B, st);
    if (rc) return bail(rc);

    // default shape: the two-column kernel where it applies and every tau is
    // 1 (as for a single handle), 64 columns per CTA for 16-bit storage and
    // 128 for FP32; else the one-column kernel, 64-wide CTAs unless most
    // domains are wide; band height filling one wave of resident CTAs
    std::vector<int> widths;
    long long nodes = 0;
    for (auto* H : B->hs) {
        widths.push_back(H->G.nx);
        nodes += (long long)H->G.nx * H->G.ny;
    }
    std::nth_element(widths.begin(), widths.begin() + widths.size() / 2, widths.end());
    tf_lbm_batch_launch L{};
    const bool narrow = B->store == kStoreF16 || B->store == kStoreBF16;
    L.pipeline = B->pair_ok && B->om1 ? kPipePair : kPipeLdg;
    if (L.pipeline == kPipePair) L.block_x = narrow ? 64 : 128;
    else L.block_x = widths[widths.size() / 2] >= 1024 ? 128 : 64;
    const int occ = std::max(1, batch_occupancy(B, L.block_x, L.pipeline));
    L.rows = rows_for_slots(B, L.block_x, (long long)occ * sm_count());
    L.graph_chunk = nodes <= (1LL << 20) ? 64 : 0;
    L.queue = 0;
    if ((rc = apply_launch(B, L, st))) return bail(rc);
    *out = B;
    return TF_LBM_OK;
}

int32_t tf_lbm_batch_items(const tf_lbm_batch* B) { return B ? B->nitems : -1; }

int tf_lbm_batch_get_launch(const tf_lbm_batch* B, tf_lbm_batch_launch* out)
{
    if (!B || !out) return TF_LBM_ERR_ARG;
    *out = B->L;
    return TF_LBM_OK;
}

int tf_lbm_batch_set_launch(tf_lbm_batch* B, const tf_lbm_batch_launch* in)
{
    if (!B) return bfail(nullptr, TF_LBM_ERR_ARG, "batch is NULL");
    int rc = validate_batch_launch(B, in);
    if (rc) return rc;
    // the work-item table is rewritten in place: let launches that read it finish
    BCK(B, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return apply_launch(B, *in, nullptr);
}

int tf_lbm_batch_step(tf_lbm_batch* B, int64_t nsteps, void* stream)
{
    if (!B) return bfail(nullptr, TF_LBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(B, TF_LBM_ERR_ARG, "nsteps must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sync_table(B, st);
    if (rc) return rc;
    const int chunk = B->L.graph_chunk;
    while (nsteps > 0) {
        if (chunk > 0 && nsteps >= chunk) {
            cudaGraphExec_t& ex = B->exec[B->phase];
            if (!ex) {
                if (!B->cap) BCK(B, cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "cudaStreamCreate");
                BCK(B, cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
                cudaError_t le = cudaSuccess;
                for (int i = 0; i < chunk && le == cudaSuccess; ++i) le = launch_batch(B, B->phase ^ (i & 1), B->cap);
                cudaGraph_t g = nullptr;
                cudaError_t ce = cudaStreamEndCapture(B->cap, &g);
                if (le != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return bcuda(B, le, "batched step (capture)");
                }
                if (ce != cudaSuccess) return bcuda(B, ce, "cudaStreamEndCapture");
                cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) {
                    ex = nullptr;
                    return bcuda(B, ie, "cudaGraphInstantiate");
                }
            }
            BCK(B, cudaGraphLaunch(ex, st), "cudaGraphLaunch");
            for (auto* H : B->hs) H->time += chunk;  // chunk is even: buffer indices unchanged
            nsteps -= chunk;
        } else {
            BCK(B, launch_batch(B, B->phase, st), "batched step");
            B->phase ^= 1;
            for (auto* H : B->hs) {
                H->cur ^= 1;
                ++H->time;
            }
            --nsteps;
        }
    }
    return TF_LBM_OK;
}

int tf_lbm_batch_tune(tf_lbm_batch* B, int32_t trial_steps, tf_lbm_batch_launch* best, void* stream)
{
    if (!B) return bfail(nullptr, TF_LBM_ERR_ARG, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sync_table(B, st);
    if (rc) return rc;
    const int steps = trial_steps <= 0 ? 16 : (trial_steps + 1) / 2 * 2;
    const int sms = sm_count();
    int ymax = 1;
    for (auto* H : B->hs) ymax = std::max(ymax, H->G.ny);

    std::vector<tf_lbm_batch_launch> cands;
    for (int pipe : {kPipePair, kPipeLdg}) {
        if (pipe == kPipePair && !B->pair_ok) continue;
        for (int bx : {64, 128, 256}) {
            const int occ = std::max(1, batch_occupancy(B, bx, pipe));
            std::vector<int> rows;
            for (int w = 1; w <= 3; ++w) rows.push_back(rows_for_slots(B, bx, (long long)w * occ * sms));
            for (int r : {8, 16, 32, 64, 128, 256}) rows.push_back(std::min(r, ymax));
            for (int r : rows)
                for (int q : {0, 1}) {
                    bool dup = false;
                    for (auto& c : cands) dup |= c.block_x == bx && c.rows == r && c.queue == q && c.pipeline == pipe;
                    if (!dup) cands.push_back(tf_lbm_batch_launch{bx, r, B->L.graph_chunk, q, pipe});
                }
        }
    }

    // copy every state aside
    std::vector<size_t> off;
    size_t total = 0;
    for (auto* H : B->hs) {
        off.push_back(total);
        total += ((size_t)H->G.plane * (H->esize + 8 * H->msize) + 255) / 256 * 256;
    }
    char* snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, total);
    if (e != cudaSuccess) return bcuda(B, e, "cudaMalloc tuning snapshot");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const tf_lbm_batch_launch old = B->L;
    auto copy_states = [&](bool out_of_handles) {
        cudaError_t r = cudaSuccess;
        for (size_t d = 0; d < B->hs.size() && r == cudaSuccess; ++d) {
            tf_lbm_handle* H = B->hs[d];
            const size_t bytes = (size_t)H->G.plane * (H->esize + 8 * H->msize);
            r = out_of_handles ? cudaMemcpyAsync(snap + off[d], H->buf[H->cur], bytes, cudaMemcpyDeviceToDevice, st)
                               : cudaMemcpyAsync(H->buf[H->cur], snap + off[d], bytes, cudaMemcpyDeviceToDevice, st);
        }
        return r;
    };
    auto finish = [&](int code) {
        cudaError_t r = copy_states(false);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(snap);
        if (code == TF_LBM_OK && r != cudaSuccess) return bcuda(B, r, "restoring the states after tuning");
        return code;
    };
    if ((e = copy_states(true)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess)
        return finish(bcuda(B, e, "tuning setup"));

    auto time_one = [&](const tf_lbm_batch_launch& c, float* ms) -> int {
        int r = apply_launch(B, c, st);
        if (r) return r;
        return time_batch(B, steps, st, e0, e1, ms);
    };
    const int k = pick_fastest(cands, time_one, &rc);
    const tf_lbm_batch_launch chosen = k >= 0 ? cands[k] : old;
    const int rc2 = apply_launch(B, rc ? old : chosen, st);
    if (rc) return finish(rc);
    if (rc2) return finish(rc2);
    if (best) *best = B->L;
    return finish(TF_LBM_OK);
}

int tf_lbm_batch_diagnostics(tf_lbm_batch* B, double h_wet, int32_t mode_x, int32_t mode_y, void* out,
                             void* stream)
{
    if (!B) return bfail(nullptr, TF_LBM_ERR_ARG, "batch is NULL");
    if (!out) return bfail(B, TF_LBM_ERR_ARG, "out must not be NULL");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return bfail(B, TF_LBM_ERR_ARG, "out must be device or managed memory");
    }
    if (isnan(h_wet)) return bfail(B, TF_LBM_ERR_ARG, "h_wet is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sync_table(B, st);
    if (rc) return rc;
    BCK(B, aux_diag(B->store, B->doms, (int)B->hs.size(), B->phase, h_wet, mode_x, mode_y, B->dpart,
                    kDiagBlocksPerDomain, (double*)out, st),
        "diagnostics kernels");
    return TF_LBM_OK;
}

}  // extern "C"
