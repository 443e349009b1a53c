// fire_local_energy_static: the local energy for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code that
// runs inside another runtime's memory pool or allocator hooks, plug-ins
// loaded into a host application that owns all device allocations, or code
// paths that must not allocate once set up.  This entry point takes the same
// inputs and outputs as fire_local_energy but uses, as its workspace, one
// file-scope device array of FIRE_STATIC_WORKSPACE_BYTES that every GPU
// which loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "../../include/fire.h"

namespace fire {
void set_last_error(const char* stage, const char* msg);
void set_single_stream(bool on);
}

// The static workspace.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_ws[FIRE_STATIC_WORKSPACE_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ws_ptr[kMaxDevices];
bool g_ws_ready[kMaxDevices];

// Set-up, once per device, with that device current: the device address of
// the static workspace.
int static_ws(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FIRE_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ws_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || p == nullptr) {
      fire::set_last_error("static workspace", cudaGetErrorString(e));
      return FIRE_ERR_CUDA;
    }
    g_ws_ptr[dev] = p;
    g_ws_ready[dev] = true;
  }
  *out = g_ws_ptr[dev];
  return FIRE_OK;
}

}  // namespace

extern "C" int fire_local_energy_static(const fire_system_t* sys, const fire_arch_t* arch,
                                        const fire_params_t* params, int64_t n_walkers, const double* r,
                                        int32_t k_cap, int32_t precision, double* e_loc, double* logabs,
                                        double* sign, double* e_kin, double* e_pot, fire_info_t* info,
                                        void* stream) {
  const size_t need = fire_workspace_size(sys, arch, n_walkers, precision, k_cap, FIRE_OP_LOCAL_ENERGY);
  if (need == 0) return FIRE_ERR_INVALID_ARG;
  if (need > (size_t)FIRE_STATIC_WORKSPACE_BYTES) {
    char msg[160];
    snprintf(msg, sizeof(msg), "needs %zu bytes of scratch, the static workspace holds %zu bytes", need,
             (size_t)FIRE_STATIC_WORKSPACE_BYTES);
    fire::set_last_error("fire_local_energy_static", msg);
    return FIRE_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  int rc = static_ws(&ws);
  if (rc) return rc;
  // The pipeline clears its status word at the start of every call; every
  // other buffer is written before it is read.  Every kernel runs on the
  // caller's stream (no second stream or event is created for this call).
  fire::set_single_stream(true);
  rc = fire_local_energy(sys, arch, params, n_walkers, r, k_cap, precision, e_loc, logabs, sign, e_kin, e_pot, info,
                         ws, (size_t)FIRE_STATIC_WORKSPACE_BYTES, stream);
  fire::set_single_stream(false);
  return rc;
}
