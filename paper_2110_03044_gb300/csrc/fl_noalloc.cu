// fl_noalloc.cu -- fl_step_rk_noalloc: the explicit step for callers that
// cannot allocate device memory.
//
// Some hosts of this library own every byte of device memory themselves: a
// solver framework that hands plugins a fixed pool and forbids them from
// calling cudaMalloc, a real-time loop that cannot afford the device-wide
// synchronisation and unbounded latency of an allocation, or a deployment that
// sizes all memory at start-up and must not grow afterwards.  Such callers can
// pass their fields but no workspace.  This entry point runs the same stage
// kernels as fl_step_rk and takes its scratch (the RK stage buffers) from a
// fixed area that is part of the library image itself.
//
// The area is a file-scope __device__ array of FL_NOALLOC_SCRATCH_BYTES;
// every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device (with that device current) asks the runtime for the address
// with cudaGetSymbolAddress and remembers it, together with the identity of
// the CUDA context it belongs to.  That first call should therefore come
// before any stream capture.  If the context changes (cudaDeviceReset, or a
// primary context released and created again), the module is loaded anew at
// another address: the next call sees the new context identity and looks the
// address up again instead of handing the kernels a stale pointer.
//
// All calls share the one area and it keeps whatever the last call left in
// it.  Nothing in it has to start at zero: every element a stage reads was
// written earlier in the same call.  Calls whose GPU work overlaps (different
// streams, or host threads that do not order their streams) race on the area;
// callers must order them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fl_internal.h"
#include "fl_kernels.h"
#include "fl_unstructured.h"

namespace fl {
// defined in fl_api.cu
fl_status check_buffer(const void *p, size_t bytes, const char *name);
fl_status check_mesh(const fl_mesh *m);
fl_status check_enums(int lim, fl_dtype dt);
size_t step_stage_bytes(const fl_mesh *m, fl_dtype dt, int rk);
}  // namespace fl

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context the address belongs to

// Device address of the scratch area on the current device: looked up on the
// first call per device, and again whenever the current context is not the
// one the cached address was taken in.
fl_status scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices)
    return fl::fail(FL_EUNSUPPORTED, "device ordinal %d out of range", device);
  unsigned long long ctx = 0;
  if (!fl::current_context_id(&ctx))
    return fl::fail(FL_ECUDA, "no CUDA context is current for device %d", device);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[device] == nullptr || g_scratch_ctx[device] != ctx) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fl::cuda_fail(e, "cudaGetSymbolAddress(scratch area)");
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_addr[device];
  return FL_OK;
}

}  // namespace

using namespace fl;

extern "C" fl_status fl_step_rk_noalloc(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                        double dtime, int64_t nsteps, void *theta,
                                        const void *u_f, void *stream) {
  fl_status st = check_mesh(m);
  if (st != FL_OK) return st;
  // check_mesh made sure the mesh's device is current; binding it again makes
  // its primary context current on this thread, so the buffer checks below
  // never need a context-creating runtime call
  if (cudaSetDevice(m->device) != cudaSuccess) return fail(FL_ECUDA, "cudaSetDevice failed");
  if ((st = check_enums(lim, dt)) != FL_OK) return st;
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (nsteps < 0) return fail(FL_EINVAL, "nsteps < 0");
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  const size_t es = dsize(dt);
  if ((st = check_buffer(theta, m->C * es, "theta")) != FL_OK) return st;
  if ((st = check_buffer(u_f, m->F * es, "u_f")) != FL_OK) return st;
  // the stage buffers only: this entry point runs without the pre-scaled
  // velocity buffer of fl_step_rk
  const size_t need = step_stage_bytes(m, dt, rk);
  if (need > (size_t)FL_NOALLOC_SCRATCH_BYTES)
    return fail(FL_EINVAL,
                "mesh needs %zu bytes of scratch but the built-in area holds %zu; "
                "use fl_step_rk with a caller-provided workspace",
                need, (size_t)FL_NOALLOC_SCRATCH_BYTES);
  if (nsteps == 0 || m->C == 0) return FL_OK;
  void *ws = nullptr;
  if ((st = scratch_address(m->device, &ws)) != FL_OK) return st;
  cudaStream_t s = as_stream(stream);
  if (m->kind == 1) return unstruct_step(m, lim, dt, rk, dtime, nsteps, theta, u_f, ws, s);
  if (line_resident_takes(m, dt)) {
    cudaError_t e = line_resident(m, lim, dt, theta, u_f, nsteps, rk, dtime, s);
    if (e != cudaSuccess) return cuda_fail(e, "1D resident kernel");
    return FL_OK;
  }
  char *wsb = static_cast<char *>(ws);
  void *A = wsb;
  void *B = wsb + align256((size_t)m->C * es);
  const cudaError_t e = struct_step(m, lim, dt, rk, dtime, nsteps, theta, u_f, A, B, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(e, "structured stage kernel");
  return FL_OK;
}
