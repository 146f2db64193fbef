// Test probe (not part of the library): runs building blocks of the stage
// kernels on arrays -- FT<double>::quot and FT<float>::quot (the van Leer
// quotient by Newton-Raphson) beside CUDA's IEEE divisions __ddiv_rn and
// __fdiv_rn, smart_piece (SMART's exact integer piece test), and
// FT<double>::sub_exact (exact differences on the integer pipe) beside
// __dsub_rn.
#include <cuda_runtime.h>

#include "fl_face.cuh"

namespace {

__global__ void k_quot(const double *n, const double *s, double *q, double *ref, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  q[i] = fl::FT<double>::quot(n[i], s[i], true);
  ref[i] = __ddiv_rn(n[i], s[i]);
}

__global__ void k_quot32(const float *n, const float *s, float *q, float *ref, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  q[i] = fl::FT<float>::quot(n[i], s[i], true);
  ref[i] = __fdiv_rn(n[i], s[i]);
}

__global__ void k_smart(const double *p, const double *q, int *piece, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  using F = fl::FT<double>;
  piece[i] = fl::smart_piece<double>(F::bits(p[i]), F::bits(q[i]), true);
}

// van Leer's paired-FP32 quotient and SMART's integer middle piece, as the
// bit patterns the limiter uses (inputs p, q > 0 as doubles)
__global__ void k_vl_ff(const double *p, const double *q, unsigned long long *g, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  using F = fl::FT<double>;
  g[i] = F::vl_quot(F::bits(p[i]), F::bits(q[i]));
}

__global__ void k_smart_mid(const double *p, const double *q, unsigned long long *g, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  using F = fl::FT<double>;
  g[i] = F::smart_mid(F::bits(p[i]), F::bits(q[i]));
}

__global__ void k_sub_exact(const double *a, const double *b, double *d, double *ref,
                            int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  d[i] = fl::FT<double>::sub_exact(a[i], b[i]);
  ref[i] = __dsub_rn(a[i], b[i]);
}

template <class T>
int to_device(const T *h, T **d, int count) {
  if (cudaMalloc(d, sizeof(T) * (size_t)count) != cudaSuccess) return 1;
  if (h && cudaMemcpy(*d, h, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice) != cudaSuccess)
    return 1;
  return 0;
}

}  // namespace

// n, s: inputs; q: quot(n, s); ref: __ddiv_rn(n, s).  Host arrays of count.
extern "C" int probe_quot(const double *n, const double *s, double *q, double *ref, int count) {
  double *dn = nullptr, *ds = nullptr, *dq = nullptr, *dr = nullptr;
  int rc = to_device(n, &dn, count) | to_device(s, &ds, count) |
           to_device<double>(nullptr, &dq, count) | to_device<double>(nullptr, &dr, count);
  if (rc == 0) {
    k_quot<<<(count + 255) / 256, 256>>>(dn, ds, dq, dr, count);
    rc = cudaMemcpy(q, dq, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
    rc |= cudaMemcpy(ref, dr, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
  }
  cudaFree(dn);
  cudaFree(ds);
  cudaFree(dq);
  cudaFree(dr);
  return rc;
}

// The same for FT<float>::quot against __fdiv_rn.
extern "C" int probe_quot32(const float *n, const float *s, float *q, float *ref, int count) {
  float *dn = nullptr, *ds = nullptr, *dq = nullptr, *dr = nullptr;
  int rc = to_device(n, &dn, count) | to_device(s, &ds, count) |
           to_device<float>(nullptr, &dq, count) | to_device<float>(nullptr, &dr, count);
  if (rc == 0) {
    k_quot32<<<(count + 255) / 256, 256>>>(dn, ds, dq, dr, count);
    rc = cudaMemcpy(q, dq, sizeof(float) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
    rc |= cudaMemcpy(ref, dr, sizeof(float) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
  }
  cudaFree(dn);
  cudaFree(ds);
  cudaFree(dq);
  cudaFree(dr);
  return rc;
}

// p, q > 0: inputs; piece: smart_piece(p, q).  Host arrays of count.
extern "C" int probe_smart(const double *p, const double *q, int *piece, int count) {
  double *dp = nullptr, *dq = nullptr;
  int *dk = nullptr;
  int rc = to_device(p, &dp, count) | to_device(q, &dq, count) | to_device<int>(nullptr, &dk, count);
  if (rc == 0) {
    k_smart<<<(count + 255) / 256, 256>>>(dp, dq, dk, count);
    rc = cudaMemcpy(piece, dk, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
  }
  cudaFree(dp);
  cudaFree(dq);
  cudaFree(dk);
  return rc;
}

// g: the bits of FT<double>::vl_quot (mode 0) or FT<double>::smart_mid
// (mode 1) for each (p, q).  Host arrays of count.
extern "C" int probe_limiter_term(const double *p, const double *q, unsigned long long *g,
                                  int count, int mode) {
  double *dp = nullptr, *dq = nullptr;
  unsigned long long *dg = nullptr;
  int rc = to_device(p, &dp, count) | to_device(q, &dq, count) |
           to_device<unsigned long long>(nullptr, &dg, count);
  if (rc == 0) {
    if (mode == 0)
      k_vl_ff<<<(count + 255) / 256, 256>>>(dp, dq, dg, count);
    else
      k_smart_mid<<<(count + 255) / 256, 256>>>(dp, dq, dg, count);
    rc = cudaMemcpy(g, dg, sizeof(unsigned long long) * (size_t)count, cudaMemcpyDeviceToHost) !=
         cudaSuccess;
  }
  cudaFree(dp);
  cudaFree(dq);
  cudaFree(dg);
  return rc;
}

// d = sub_exact(a, b); ref = __dsub_rn(a, b).  Host arrays of count.
extern "C" int probe_sub_exact(const double *a, const double *b, double *d, double *ref,
                               int count) {
  double *da = nullptr, *db = nullptr, *dd = nullptr, *dr = nullptr;
  int rc = to_device(a, &da, count) | to_device(b, &db, count) |
           to_device<double>(nullptr, &dd, count) | to_device<double>(nullptr, &dr, count);
  if (rc == 0) {
    k_sub_exact<<<(count + 255) / 256, 256>>>(da, db, dd, dr, count);
    rc = cudaMemcpy(d, dd, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess;
    rc |= cudaMemcpy(ref, dr, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost) !=
          cudaSuccess;
  }
  cudaFree(da);
  cudaFree(db);
  cudaFree(dd);
  cudaFree(dr);
  return rc;
}
