// Test probe (not part of the library): records a device-side error in a
// mesh's status word from a kernel, the way the library's own kernels do
// when a bounded wait gives up, so that a test can check that the next call
// on the mesh returns it.  Compiled against the library's internal header,
// which gives the mesh object's layout.
#include <cuda_runtime.h>

#include "fl_internal.h"

namespace {
__global__ void k_record(int *status, int code) { fl::record_status(status, code); }
}  // namespace

extern "C" int probe_record_status(void *mesh, int code) {
  fl_mesh *m = static_cast<fl_mesh *>(mesh);
  if (m == nullptr || m->status == nullptr) return -1;
  k_record<<<1, 1>>>(m->status, code);
  if (cudaGetLastError() != cudaSuccess) return -2;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -3;
}
