// fl_order.cu -- field order conversions of renumbered face-based meshes
// (fl_mesh_to_internal / fl_mesh_to_user), and the halo gather and scatter
// of a decomposed run (fl_halo_pack / fl_halo_unpack).
//
// FL_RENUMBER relabels cells and faces (permutations P_c, P_f) so that the
// stage kernels read compact blocks; the compute calls then work on fields
// in that internal order.  A caller holding fields in its own numbering
// converts them here, once before and once after a rollout: one launch that
// gathers (to user order) or scatters (to internal order) through the
// mesh's device copy of the permutation.  Reads of src and writes of dst are
// coalesced on the user-indexed side; the other side is a permuted access.
#include <cuda_runtime.h>

#include "fl_internal.h"

namespace fl {
fl_status check_buffer(const void *p, size_t bytes, const char *name);
fl_status check_mesh(const fl_mesh *m);
}  // namespace fl

namespace {

// to_internal: dst[perm[i]] = src[i]; to_user: dst[i] = src[perm[i]]
// (perm[i] = internal index of user index i; a permutation, so the scatter
// writes every element of dst exactly once)
template <class T, bool TO_INTERNAL>
__global__ void k_reorder(const T *__restrict__ src, T *__restrict__ dst,
                          const int32_t *__restrict__ perm, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = perm[i];
    if (TO_INTERNAL)
      dst[j] = src[i];
    else
      dst[i] = src[j];
  }
}

template <bool TO_INTERNAL>
fl_status reorder(const fl_mesh *m, fl_field_kind kind, fl_dtype dt, const void *src, void *dst,
                  void *stream) {
  using namespace fl;
  fl_status st = check_mesh(m);
  if (st != FL_OK) return st;
  if (kind != FL_FIELD_CELL && kind != FL_FIELD_FACE)
    return fail(FL_EINVAL, "unknown field kind %d", (int)kind);
  if (dt != FL_F32 && dt != FL_F64) return fail(FL_EINVAL, "unknown dtype %d", (int)dt);
  const long long n = kind == FL_FIELD_CELL ? m->C : m->F;
  const size_t bytes = (size_t)n * dsize(dt);
  if ((st = check_buffer(src, bytes, "src")) != FL_OK) return st;
  if ((st = check_buffer(dst, bytes, "dst")) != FL_OK) return st;
  const char *s0 = static_cast<const char *>(src), *d0 = static_cast<const char *>(dst);
  if (n > 0 && s0 < d0 + bytes && d0 < s0 + bytes)
    return fail(FL_EINVAL, "src and dst overlap");
  if (n == 0) return FL_OK;
  cudaStream_t s = as_stream(stream);
  const int32_t *perm = nullptr;
  if (m->kind == 1 && m->renumbered) perm = kind == FL_FIELD_CELL ? m->u.perm_cell : m->u.perm_face;
  if (perm == nullptr) {
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? FL_OK : cuda_fail(e, "field copy");
  }
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  if (dt == FL_F64)
    k_reorder<double, TO_INTERNAL><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const double *>(src), static_cast<double *>(dst), perm, n);
  else
    k_reorder<float, TO_INTERNAL><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const float *>(src), static_cast<float *>(dst), perm, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "reorder kernel");
}

// dst[i] = src[index[i]] for index[i] in [0, n_src); an index outside
// records FL_EINDEX in the mesh's status word and leaves dst[i] as it was
template <class T>
__global__ void k_halo_pack(const T *__restrict__ src, const int32_t *__restrict__ index,
                            long long n, long long n_src, T *__restrict__ dst, int *status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = index[i];
    if (j < 0 || j >= n_src) {
      fl::record_status(status, (int)FL_EINDEX);
      continue;
    }
    dst[i] = src[j];
  }
}

// dst[index[i]] = src[i] for index[i] in [0, n_dst); an index outside
// records FL_EINDEX and writes nothing
template <class T>
__global__ void k_halo_unpack(const T *__restrict__ src, const int32_t *__restrict__ index,
                              long long n, long long n_dst, T *__restrict__ dst, int *status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = index[i];
    if (j < 0 || j >= n_dst) {
      fl::record_status(status, (int)FL_EINDEX);
      continue;
    }
    dst[j] = src[i];
  }
}

}  // namespace

extern "C" {

fl_status fl_halo_unpack(const fl_mesh *mesh, fl_dtype dtype, const void *src,
                         const int32_t *index, int64_t n, void *dst, void *stream) {
  using namespace fl;
  fl_status st = check_mesh(mesh);
  if (st != FL_OK) return st;
  if (dtype != FL_F32 && dtype != FL_F64) return fail(FL_EINVAL, "unknown dtype %d", (int)dtype);
  if (n < 0) return fail(FL_EINVAL, "n < 0");
  if (n == 0) return FL_OK;
  const size_t es = dsize(dtype);
  if ((st = check_buffer(src, (size_t)n * es, "src")) != FL_OK) return st;
  if ((st = check_buffer(index, (size_t)n * sizeof(int32_t), "index")) != FL_OK) return st;
  if ((st = check_buffer(dst, (size_t)mesh->C * es, "dst")) != FL_OK) return st;
  const char *s0 = static_cast<const char *>(src), *d0 = static_cast<const char *>(dst);
  const size_t sb = (size_t)n * es, db = (size_t)mesh->C * es;
  if (s0 < d0 + db && d0 < s0 + sb) return fail(FL_EINVAL, "src and dst overlap");
  cudaStream_t s = as_stream(stream);
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  if (dtype == FL_F64)
    k_halo_unpack<double><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const double *>(src), index, n, mesh->C, static_cast<double *>(dst),
        mesh->status);
  else
    k_halo_unpack<float><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const float *>(src), index, n, mesh->C, static_cast<float *>(dst),
        mesh->status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "halo unpack kernel");
}

fl_status fl_halo_pack(const fl_mesh *mesh, fl_dtype dtype, const void *src, const int32_t *index,
                       int64_t n, void *dst, void *stream) {
  using namespace fl;
  fl_status st = check_mesh(mesh);
  if (st != FL_OK) return st;
  if (dtype != FL_F32 && dtype != FL_F64) return fail(FL_EINVAL, "unknown dtype %d", (int)dtype);
  if (n < 0) return fail(FL_EINVAL, "n < 0");
  if (n == 0) return FL_OK;
  const size_t es = dsize(dtype);
  if ((st = check_buffer(src, (size_t)mesh->C * es, "src")) != FL_OK) return st;
  if ((st = check_buffer(index, (size_t)n * sizeof(int32_t), "index")) != FL_OK) return st;
  if ((st = check_buffer(dst, (size_t)n * es, "dst")) != FL_OK) return st;
  const char *s0 = static_cast<const char *>(src), *d0 = static_cast<const char *>(dst);
  const size_t sb = (size_t)mesh->C * es, db = (size_t)n * es;
  if (s0 < d0 + db && d0 < s0 + sb) return fail(FL_EINVAL, "src and dst overlap");
  cudaStream_t s = as_stream(stream);
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  if (dtype == FL_F64)
    k_halo_pack<double><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const double *>(src), index, n, mesh->C, static_cast<double *>(dst),
        mesh->status);
  else
    k_halo_pack<float><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const float *>(src), index, n, mesh->C, static_cast<float *>(dst),
        mesh->status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "halo pack kernel");
}

fl_status fl_mesh_to_internal(const fl_mesh *mesh, fl_field_kind kind, fl_dtype dtype,
                              const void *src, void *dst, void *stream) {
  return reorder<true>(mesh, kind, dtype, src, dst, stream);
}

fl_status fl_mesh_to_user(const fl_mesh *mesh, fl_field_kind kind, fl_dtype dtype,
                          const void *src, void *dst, void *stream) {
  return reorder<false>(mesh, kind, dtype, src, dst, stream);
}

}  // extern "C"
