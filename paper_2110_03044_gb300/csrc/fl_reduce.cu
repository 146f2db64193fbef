// fl_reduce.cu -- the generalised reduction (kred, Section 3.2): maximum of
// |x| (for the CFL step size) and the conserved total sum_c V_c theta_c, both
// flagging NaN / Inf.  Two passes: per-CTA partials into the caller's
// workspace, then one CTA folds them.  The sum is compensated (Neumaier) and
// partials are merged with exact two-sums, so the result does not depend on
// the order in which CTAs finish.
#include <cuda_runtime.h>

#include <cmath>

#include "fl_internal.h"
#include "fl_kernels.h"

namespace fl {

namespace {

constexpr int RB = 256;      // threads per CTA
constexpr int RMAXB = 1024;  // partial slots

struct Partial {
  double s, c;   // sum and compensation (or max in s)
  int nonfinite;
  int pad;
};

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void merge_sum(double &s, double &c, double s2, double c2) {
  double t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __dadd_rn(c, __dadd_rn(c2, e));
}

template <int MODE, class T>  // MODE 0: max |x|, 1: sum V x
__global__ void __launch_bounds__(RB) k_reduce(const T *x, const double *vol, double vconst,
                                               long long n, Partial *part) {
  double s = 0.0, c = 0.0;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)RB + threadIdx.x; i < n; i += (long long)gridDim.x * RB) {
    const double v = (double)x[i];
    bad |= !isfinite(v);
    if (MODE == 0) {
      s = fmax(s, fabs(v));
    } else {
      const double w = vol ? vol[i] : vconst;
      double t, e;
      two_sum(s, __dmul_rn(w, v), t, e);
      s = t;
      c = __dadd_rn(c, e);
    }
  }
  __shared__ double ss[RB], sc[RB];
  __shared__ int sb[RB];
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      if (MODE == 0) {
        ss[threadIdx.x] = fmax(ss[threadIdx.x], ss[threadIdx.x + w]);
      } else {
        double a = ss[threadIdx.x], ac = sc[threadIdx.x];
        merge_sum(a, ac, ss[threadIdx.x + w], sc[threadIdx.x + w]);
        ss[threadIdx.x] = a;
        sc[threadIdx.x] = ac;
      }
      sb[threadIdx.x] |= sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x].s = ss[0];
    part[blockIdx.x].c = sc[0];
    part[blockIdx.x].nonfinite = sb[0];
  }
}

template <int MODE>
__global__ void __launch_bounds__(RB) k_reduce_final(Partial *part, int nb, Partial *out) {
  __shared__ double ss[RB], sc[RB];
  __shared__ int sb[RB];
  double s = 0.0, c = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < nb; i += RB) {
    if (MODE == 0) s = fmax(s, part[i].s);
    else merge_sum(s, c, part[i].s, part[i].c);
    bad |= part[i].nonfinite;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      if (MODE == 0) {
        ss[threadIdx.x] = fmax(ss[threadIdx.x], ss[threadIdx.x + w]);
      } else {
        double a = ss[threadIdx.x], ac = sc[threadIdx.x];
        merge_sum(a, ac, ss[threadIdx.x + w], sc[threadIdx.x + w]);
        ss[threadIdx.x] = a;
        sc[threadIdx.x] = ac;
      }
      sb[threadIdx.x] |= sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->s = ss[0];
    out->c = sc[0];
    out->nonfinite = sb[0];
  }
}

template <int MODE>
cudaError_t run(fl_dtype dt, const void *x, const double *vol, double vconst, int64_t n, void *ws,
                cudaStream_t st, double *out, int *nonfinite) {
  Partial *part = static_cast<Partial *>(ws);
  Partial *fin = part + RMAXB;
  long long nb = (n + RB - 1) / RB;
  if (nb > RMAXB) nb = RMAXB;
  if (nb < 1) nb = 1;
  if (dt == FL_F64)
    k_reduce<MODE, double><<<(unsigned)nb, RB, 0, st>>>(static_cast<const double *>(x), vol, vconst,
                                                        n, part);
  else
    k_reduce<MODE, float><<<(unsigned)nb, RB, 0, st>>>(static_cast<const float *>(x), vol, vconst,
                                                       n, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<MODE><<<1, RB, 0, st>>>(part, (int)nb, fin);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Partial h;
  e = cudaMemcpyAsync(&h, fin, sizeof(Partial), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *out = (MODE == 0) ? h.s : h.s + h.c;
  *nonfinite = h.nonfinite;
  return cudaSuccess;
}

}  // namespace

size_t reduce_ws_bytes() { return align256(sizeof(Partial) * (RMAXB + 1)); }

cudaError_t reduce_max_abs(fl_dtype dt, const void *x, int64_t n, void *ws, cudaStream_t st,
                           double *out, int *nonfinite) {
  return run<0>(dt, x, nullptr, 0.0, n, ws, st, out, nonfinite);
}

cudaError_t reduce_mass(fl_dtype dt, const void *theta, const double *vol, double vconst, int64_t n,
                        void *ws, cudaStream_t st, double *out, int *nonfinite) {
  return run<1>(dt, theta, vol, vconst, n, ws, st, out, nonfinite);
}

}  // namespace fl
