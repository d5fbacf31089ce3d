// xy_noalloc.cu -- xy_sweep_noalloc: the fused sweep without any allocation.
//
// Some callers cannot allocate device memory at the moment they want to run
// sweeps: a process whose device memory is all handed to its own caching
// allocator, code that cannot afford the device-wide synchronisation that
// cudaFree implies, or a run that must not be able to fail with an
// out-of-memory error half way.  For them this entry point runs the same fused
// kernel as xy_sweep, with the second (ping-pong) lattice buffer the kernel
// needs taken from a fixed array in this file instead of from cudaMalloc.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocMaxL^2 floats, 4 MiB) until the process exits.  In
// host code its name is only a host-side stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "xy.h"
#include "xy_internal.h"

namespace {

constexpr int kNoAllocMaxL = 1024;
constexpr int kMaxDevices = 64;

// The ping-pong buffer shared by every call on a device.
static __device__ __align__(256) float g_noalloc_pong[(size_t)kNoAllocMaxL * kNoAllocMaxL];

std::mutex g_setup_mu;
float* g_pong_ptr[kMaxDevices] = {};

// Device address of g_noalloc_pong on the current device (set up once per device).
cudaError_t pong_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_pong_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_pong);
    if (e != cudaSuccess) return e;
    g_pong_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_pong_ptr[dev];
  return cudaSuccess;
}

thread_local char g_msg[256] = "no error";

xy_status fail(xy_status st, const char* what) {
  (void)cudaGetLastError();   // leave no non-sticky error behind for later launch checks
  snprintf(g_msg, sizeof(g_msg), "xy_sweep_noalloc: %s", what);
  return st;
}

}  // namespace

extern "C" {

xy_status xy_sweep_noalloc(const xy_params* p, float* d_angles, uint32_t first_sweep,
                           int64_t n_sweeps, xy_record* d_records, void* cuda_stream) {
  xyk::NvtxRange range("xy_sweep_noalloc");
  if (!p || !d_angles || n_sweeps < 0 || (n_sweeps > 0 && !d_records))
    return fail(XY_EINVAL, "NULL pointer or negative sweep count");
  if (p->L < 128 || p->L > kNoAllocMaxL || (p->L % 128) != 0)
    return fail(XY_EINVAL, "L must be a multiple of 128 and at most 1024 (the fixed buffer)");
  if (!(p->beta >= 0.0) || !isfinite(p->beta) || !isfinite(p->J) || !(p->delta > 0.0) ||
      p->delta > M_PI + 1e-12 || p->sincos_mode < 0 || p->sincos_mode > 2 ||
      p->reduce_mode < 0 || p->reduce_mode > 1)
    return fail(XY_EINVAL, "bad beta, J, delta, sincos_mode or reduce_mode");
  if ((uint64_t)first_sweep + (uint64_t)n_sweeps > 0xffffffffull)
    return fail(XY_EINVAL, "sweep counter would pass 2^32 - 1");
  if (reinterpret_cast<uintptr_t>(d_angles) & 15u) return fail(XY_EINVAL, "d_angles not 16-byte aligned");
  if (n_sweeps == 0) return XY_OK;

  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  float* pong = nullptr;
  cudaError_t e = pong_address(&pong);
  if (e != cudaSuccess) return fail(XY_ECUDA, cudaGetErrorString(e));

  // records accumulate with atomics: they must start at zero
  e = cudaMemsetAsync(d_records, 0, (size_t)n_sweeps * sizeof(xy_record), stream);
  if (e != cudaSuccess) return fail(XY_ECUDA, cudaGetErrorString(e));

  // the tile kernel's staged rows come by TMA: tensor maps of both buffers
  xyk::FusedMaps maps;
  if (!xyk::encode_fused_maps(&maps, d_angles, pong, p->L))
    return fail(XY_ECUDA, "tensor maps of the state buffers could not be encoded");

  xyk::FusedArgs a;
  a.maps = &maps;
  a.L = p->L;
  a.W = p->L / 2;
  a.K = (float)(p->beta * p->J);
  a.delta = (float)p->delta;
  a.rk = xyd::make_round_keys(p->seed);
  a.lattice_id = p->lattice_id;
  a.beta = p->beta;
  float* cur = d_angles;
  float* nxt = pong;
  for (int64_t i = 0; i < n_sweeps; ++i) {
    a.src = cur;
    a.dst = nxt;
    a.sweep = first_sweep + (uint32_t)i;
    a.rec = d_records + i;
    e = xyk::launch_fused_sweep(p->sincos_mode, p->reduce_mode, a, stream);
    if (e != cudaSuccess) return fail(XY_ECUDA, cudaGetErrorString(e));
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != d_angles) {
    e = cudaMemcpyAsync(d_angles, cur, (size_t)p->L * p->L * sizeof(float),
                        cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return fail(XY_ECUDA, cudaGetErrorString(e));
  }
  return XY_OK;
}

const char* xy_noalloc_last_error(void) { return g_msg; }

}  // extern "C"
