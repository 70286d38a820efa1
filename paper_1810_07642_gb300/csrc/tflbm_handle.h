// Internal definition of the opaque tf_lbm_handle, shared by the C-ABI
// translation units (tflbm_api.cu, tflbm_adjoint.cu).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tflbm.h"
#include "tflbm_internal.h"

using namespace tflbm;

struct tf_lbm_handle {
    tf_lbm_params p;
    int device = 0;
    size_t esize = 4;          // bytes of the compute type (plane 0, fields)
    size_t msize = 4;          // bytes of one stored moving population
    bool dbl = false;          // compute type is double
    StoreDesc desc{};          // storage encoding (for the auxiliary kernels)
    Geom G{};
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;               // buf[cur] holds the post-collision populations of step t-1
    void* kappa = nullptr;     // [ny][nx] or null (uniform)
    double kappa_u = 0.0;
    double href = 0.0;         // reference height (exactly representable in the storage type)
    double* partials = nullptr;
    double* result = nullptr;
    int nmass = 0;
    int* flag = nullptr;
    int* status = nullptr;     // device word kernels set (kStatusTimeout)
    int wait_limit = kWaitLimit;  // polls of one mbarrier before a bulk-copy kernel gives up
    void* diag = nullptr;      // 2 * ny * nx scratch for tf_lbm_pressure_force (lazy)
    int64_t time = 0;
    Shape shape{128, 64, kPipeLdg};  // replaced by the occupancy-derived default in tf_lbm_init
    int graph_chunk = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::string err;
    void* adj = nullptr;       // adjoint scratch (lazy): 10 fields of the compute type
    void* dscr = nullptr;      // diagnostics scratch (lazy): one BatchDomain entry + partial sums
    void* tscr = nullptr;      // term-norm scratch (lazy): 5 fields + partial sums
};


namespace tflbm {
// Per-run step constants of a handle, in the compute type T.
template <typename T>
Consts<T> make_consts(const tf_lbm_handle* H);
// Launch one fused step from buf[from] into buf[from ^ 1].
cudaError_t launch_one_step(tf_lbm_handle* H, int from, cudaStream_t st);
// Launch one fused step between two population buffers of the handle's layout.
cudaError_t launch_step_between(tf_lbm_handle* H, const void* fin, void* fout, cudaStream_t st);
// Fused adjoint step (tflbm_adjoint_march.cuh) from the raw buffer whose pull is f(t).
cudaError_t adjoint_march_dispatch(tf_lbm_handle* H, const void* fin, const void* an, void* a, void* gk,
                                   cudaStream_t st);
// Record an error message on H (or for the calling thread when H is null).
int handle_fail(tf_lbm_handle* H, int code, const std::string& msg);
int handle_cuda_fail(tf_lbm_handle* H, cudaError_t e, const char* what);
// ARG error unless ptr is device or managed memory of the current device.
int handle_check_dev_ptr(tf_lbm_handle* H, const void* ptr, const char* name, bool allow_null);
// Forget the handle's captured step graphs (after a launch-shape change).
void handle_drop_graphs(tf_lbm_handle* H);
// Streaming multiprocessors of the current device.
int sm_count();
// Adjoint of one step (tflbm_adjoint.cu).
cudaError_t adjoint_step_dispatch(tf_lbm_handle* H, const void* f, const void* a_next, void* a,
                                  void* grad_kappa, cudaStream_t st);
}  // namespace tflbm
