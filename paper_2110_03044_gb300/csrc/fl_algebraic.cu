// fl_algebraic.cu -- the paper's algebraic implementation of the flux
// limiter, built from two kernel types only: sparse matrix-vector products
// (SpMV, ELLPACK) and generalized pointwise binary operators (kbin).
//
// Algorithm 1 (theta_f of a face-based mesh) as 4 SpMV + 4 kbin calls, with
// the upstream difference in its corrected form d_U = (Q T - S) theta
// (Section 3: S = 1/2 N (I (x) D^A) N^T E, T = 1/2 N (I (x) A) N^T E; the
// printed "+ S" holds for one flow direction only, so the matrix stored
// here is -S):
//   d   <- E theta            SpMV (|F| x |C|, 2 per row)
//   d   <- Q d                kbin signxty
//   r   <- T theta            SpMV (2k per row)
//   r   <- Q r                kbin signxty
//   r   <- r + (-S) theta     SpMV (2k per row)
//   r   <- r / d              kbin axdy
//   t_f <- F(r) d             kbin <limiter>xty, F = (Psi - 1) / 2
//   t_f <- t_f + Pi theta     SpMV (2 per row)
// and Algorithm 5's forward-Euler update theta <- theta + dt M U(u_f) t_f as
// kbin (U t_f) + SpMV (M = V^-1 E^T diag(A), k per row) + kbin (axpy).
//
// The matrices are assembled on the host from the face-cell incidence,
// normals, areas and volumes alone -- the chain never looks up an upstream
// cell -- and stored in ELLPACK with 8-byte values and 4-byte column
// indices, column-major (entry k of row r at k * rows + r) so that the
// threads of a warp read consecutive words.  Rows keep their structural
// entries (the cells of every face adjacent to f), zero coefficients
// included, as the paper's storage count does (2 |F| non-zeros for E and
// Pi, 2k |F| for S and T).  This path is the comparison baseline for the
// fused stencil kernels; it is FP64 only.
//
// Ties and degenerate cases follow the stencil path: u_f = 0, -0 and NaN
// select -1 (Table 1 signxty); d_u == 0 keeps the upwind value (the
// limiter kbin returns F(r) d = -d/2 there, so t_f = Pi theta - d/2 =
// theta_C).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "fl_face.cuh"
#include "fl_internal.h"

namespace fl {
fl_status check_buffer(const void *p, size_t bytes, const char *name);
fl_status check_enums(int lim, fl_dtype dt);
}  // namespace fl

struct fl_ell {
  int64_t rows = 0;
  int width = 0;
  double *val = nullptr;  // [width][rows]
  int32_t *col = nullptr;
  int64_t nnz = 0;        // structural entries (without the padding)
};

struct fl_alg {
  int device = 0;
  int64_t C = 0, F = 0;
  fl_ell E, Pi, T, mS, M;
};

namespace fl {
namespace {

// ------------------------------------------------------------- kernels
constexpr int AT = 256;

__device__ __forceinline__ long long gtid() {
  return blockIdx.x * (long long)blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// y = (ACC ? y : 0) + A x
template <bool ACC>
__global__ void __launch_bounds__(AT) k_ell_spmv(const double *__restrict__ val,
                                                 const int32_t *__restrict__ col, long long rows,
                                                 int width, const double *__restrict__ x,
                                                 double *__restrict__ y) {
  for (long long r = gtid(); r < rows; r += gstride()) {
    double acc = ACC ? y[r] : 0.0;
    for (int k = 0; k < width; ++k) {
      const long long e = (long long)k * rows + r;
      acc = __fma_rn(val[e], __ldg(x + col[e]), acc);
    }
    y[r] = acc;
  }
}

// signxty: y_i <- y_i (u_i > 0 ? +1 : -1)
__global__ void __launch_bounds__(AT) k_signxty(const double *__restrict__ u, double *y,
                                                long long n) {
  for (long long i = gtid(); i < n; i += gstride())
    if (!upwind_positive(u[i])) y[i] = -y[i];
}

// axdy: r_i <- r_i / d_i
__global__ void __launch_bounds__(AT) k_axdy(const double *__restrict__ d, double *r, long long n) {
  for (long long i = gtid(); i < n; i += gstride()) r[i] = __ddiv_rn(r[i], d[i]);
}

// <limiter>xty: t_i <- d_i F(r_i), F = (Psi(r) - 1) / 2; d_i == 0 gives -d_i/2
// (Psi taken as 0: the upwind value)
template <int LIM>
__device__ __forceinline__ double psi_of(double r) {
  if (LIM == LIM_UPWIND) return 0.0;
  if (LIM == LIM_CENTRAL) return 1.0;
  if (LIM == LIM_MINMOD) return fmax(0.0, fmin(1.0, r));
  if (LIM == LIM_SUPERBEE) return fmax(0.0, fmax(fmin(1.0, 2.0 * r), fmin(r, 2.0)));
  if (LIM == LIM_SMART) return fmax(0.0, fmin(fmin(2.0 * r, __fma_rn(0.75, r, 0.25)), 4.0));
  // van Leer: (r + |r|) / (1 + |r|) = 2 r / (1 + r) for r > 0, else 0; r = +inf gives 2
  if (!(r > 0.0)) return 0.0;
  if (isinf(r)) return 2.0;
  return 2.0 * __ddiv_rn(r, 1.0 + r);
}

template <int LIM>
__global__ void __launch_bounds__(AT) k_limxty(const double *__restrict__ r,
                                               const double *__restrict__ d, double *t,
                                               long long n) {
  for (long long i = gtid(); i < n; i += gstride()) {
    const double di = d[i];
    const double psi = (di == 0.0) ? 0.0 : psi_of<LIM>(r[i]);
    t[i] = di * (0.5 * (psi - 1.0));
  }
}

// phi_i <- u_i t_i (the diagonal U(u_f))
__global__ void __launch_bounds__(AT) k_uxty(const double *__restrict__ u,
                                             const double *__restrict__ t, double *phi,
                                             long long n) {
  for (long long i = gtid(); i < n; i += gstride()) phi[i] = u[i] * t[i];
}

// theta_i <- theta_i + dt R_i
__global__ void __launch_bounds__(AT) k_axpy(double dt, const double *__restrict__ R, double *th,
                                             long long n) {
  for (long long i = gtid(); i < n; i += gstride()) th[i] = __fma_rn(dt, R[i], th[i]);
}

unsigned grid_for(long long n) {
  long long b = (n + AT - 1) / AT;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

cudaError_t spmv(const fl_ell &A, const double *x, double *y, bool acc, cudaStream_t st) {
  if (A.rows == 0) return cudaSuccess;
  if (acc)
    k_ell_spmv<true><<<grid_for(A.rows), AT, 0, st>>>(A.val, A.col, A.rows, A.width, x, y);
  else
    k_ell_spmv<false><<<grid_for(A.rows), AT, 0, st>>>(A.val, A.col, A.rows, A.width, x, y);
  return cudaGetLastError();
}

cudaError_t limxty(int lim, const double *r, const double *d, double *t, long long n,
                   cudaStream_t st) {
  const unsigned g = grid_for(n);
  switch (lim) {
    case LIM_UPWIND: k_limxty<LIM_UPWIND><<<g, AT, 0, st>>>(r, d, t, n); break;
    case LIM_CENTRAL: k_limxty<LIM_CENTRAL><<<g, AT, 0, st>>>(r, d, t, n); break;
    case LIM_MINMOD: k_limxty<LIM_MINMOD><<<g, AT, 0, st>>>(r, d, t, n); break;
    case LIM_VANLEER: k_limxty<LIM_VANLEER><<<g, AT, 0, st>>>(r, d, t, n); break;
    case LIM_SUPERBEE: k_limxty<LIM_SUPERBEE><<<g, AT, 0, st>>>(r, d, t, n); break;
    case LIM_SMART: k_limxty<LIM_SMART><<<g, AT, 0, st>>>(r, d, t, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Algorithm 1 into t (|F|), with d and r (|F| each) as scratch
cudaError_t face_values(const fl_alg *a, int lim, const double *th, const double *u, double *d,
                        double *r, double *t, cudaStream_t st) {
  const long long F = a->F;
  cudaError_t e = spmv(a->E, th, d, false, st);
  if (e == cudaSuccess) {
    k_signxty<<<grid_for(F), AT, 0, st>>>(u, d, F);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = spmv(a->T, th, r, false, st);
  if (e == cudaSuccess) {
    k_signxty<<<grid_for(F), AT, 0, st>>>(u, r, F);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = spmv(a->mS, th, r, true, st);
  if (e == cudaSuccess) {
    k_axdy<<<grid_for(F), AT, 0, st>>>(d, r, F);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = limxty(lim, r, d, t, F, st);
  if (e == cudaSuccess) e = spmv(a->Pi, th, t, true, st);
  return e;
}

// ------------------------------------------------------------ assembly
template <class Fn>
void par_for(int64_t n, Fn fn) {
  unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  if (n < 20000 || nt == 1) {
    fn((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back(fn, b, e);
  }
  for (auto &x : th) x.join();
}

struct HostEll {
  int64_t rows = 0;
  int width = 0;
  int64_t nnz = 0;
  std::vector<double> val;
  std::vector<int32_t> col;
};

// Rows given as (col, val) lists, duplicates merged, ordered by column.  Two
// passes over the rows (the first sizes the rows, the second writes the
// column-major arrays), so the only large allocation is the result itself.
template <class RowFn>
HostEll build_ell(int64_t rows, RowFn row_fn) {
  HostEll H;
  H.rows = rows;
  auto merged = [&](int64_t r, std::vector<std::pair<int32_t, double>> &ent) {
    ent.clear();
    row_fn(r, ent);
    std::sort(ent.begin(), ent.end(),
              [](const auto &x, const auto &y) { return x.first < y.first; });
    size_t n = 0;
    for (size_t i = 0; i < ent.size(); ++i) {
      if (n > 0 && ent[n - 1].first == ent[i].first) ent[n - 1].second += ent[i].second;
      else ent[n++] = ent[i];
    }
    ent.resize(n);
  };
  std::vector<int> len(rows);
  par_for(rows, [&](int64_t b, int64_t e) {
    std::vector<std::pair<int32_t, double>> ent;
    for (int64_t r = b; r < e; ++r) {
      merged(r, ent);
      len[r] = (int)ent.size();
    }
  });
  int w = 0;
  int64_t nnz = 0;
  for (int64_t r = 0; r < rows; ++r) {
    w = std::max(w, len[r]);
    nnz += len[r];
  }
  H.width = w;
  H.nnz = nnz;
  H.val.assign((size_t)rows * w, 0.0);
  H.col.assign((size_t)rows * w, 0);
  par_for(rows, [&](int64_t b, int64_t e) {
    std::vector<std::pair<int32_t, double>> ent;
    for (int64_t r = b; r < e; ++r) {
      merged(r, ent);
      const int32_t pad = ent.empty() ? 0 : ent[0].first;
      for (int k = 0; k < w; ++k) {
        const bool in = k < (int)ent.size();
        H.col[(size_t)k * rows + r] = in ? ent[k].first : pad;
        H.val[(size_t)k * rows + r] = in ? ent[k].second : 0.0;
      }
    }
  });
  return H;
}

fl_status upload(const HostEll &H, fl_ell *D) {
  D->rows = H.rows;
  D->width = H.width;
  D->nnz = H.nnz;
  const size_t n = (size_t)H.rows * H.width;
  if (n == 0) return FL_OK;
  if (cudaMalloc(&D->val, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&D->col, n * sizeof(int32_t)) != cudaSuccess)
    return fail(FL_ENOMEM, "ELLPACK allocation of %zu entries failed", n);
  if (cudaMemcpy(D->val, H.val.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(D->col, H.col.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(FL_ECUDA, "ELLPACK upload failed");
  return FL_OK;
}

void free_ell(fl_ell &D) {
  if (D.val) cudaFree(D.val);
  if (D.col) cudaFree(D.col);
  D.val = nullptr;
  D.col = nullptr;
}

size_t ell_bytes(const fl_ell &D) { return (size_t)D.rows * D.width * 12; }

}  // namespace
}  // namespace fl

using namespace fl;

extern "C" {

fl_status fl_alg_create(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                        const double *normals, const double *areas, const double *volumes,
                        fl_alg **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_cells < 1 || n_faces < 0 || n_cells >= (1LL << 31) || n_faces >= (1LL << 31))
    return fail(FL_EINVAL, "need 1 <= n_cells < 2^31 and 0 <= n_faces < 2^31");
  if (n_faces > 0 && (!face_cells || !normals || !areas)) return fail(FL_EINVAL, "NULL face array");
  if (!volumes) return fail(FL_EINVAL, "NULL volumes");
  const int64_t C = n_cells, F = n_faces;
  for (int64_t f = 0; f < F; ++f) {
    const int32_t a = face_cells[2 * f], b = face_cells[2 * f + 1];
    if (a < 0 || b < 0 || a >= C || b >= C) return fail(FL_EINDEX, "face %lld: cell out of range", (long long)f);
    if (a == b) return fail(FL_EINVAL, "face %lld joins cell %d to itself", (long long)f, a);
    if (!(areas[f] > 0) || !std::isfinite(areas[f])) return fail(FL_EINVAL, "face %lld: bad area", (long long)f);
  }
  for (int64_t c = 0; c < C; ++c)
    if (!(volumes[c] > 0) || !std::isfinite(volumes[c])) return fail(FL_EINVAL, "cell %lld: bad volume", (long long)c);
  // cell -> faces (CSR)
  std::vector<int64_t> cptr(C + 1, 0);
  for (int64_t f = 0; f < F; ++f) {
    ++cptr[face_cells[2 * f] + 1];
    ++cptr[face_cells[2 * f + 1] + 1];
  }
  for (int64_t c = 0; c < C; ++c) cptr[c + 1] += cptr[c];
  std::vector<int32_t> cf(cptr[C]);
  {
    std::vector<int64_t> pos(cptr.begin(), cptr.end() - 1);
    for (int64_t f = 0; f < F; ++f) {
      cf[pos[face_cells[2 * f]]++] = (int32_t)f;
      cf[pos[face_cells[2 * f + 1]]++] = (int32_t)f;
    }
  }
  auto dotn = [&](int64_t f, int64_t j) {
    return normals[3 * f] * normals[3 * j] + normals[3 * f + 1] * normals[3 * j + 1] +
           normals[3 * f + 2] * normals[3 * j + 2];
  };
  fl_alg *a = new (std::nothrow) fl_alg();
  if (!a) return fail(FL_ENOMEM, "host allocation failed");
  cudaGetDevice(&a->device);
  a->C = C;
  a->F = F;
  fl_status s = FL_OK;
  {  // E: E[f, c0] = -1, E[f, c1] = +1 (eq. Tfc)
    HostEll H = build_ell(F, [&](int64_t f, auto &ent) {
      ent.push_back({face_cells[2 * f], -1.0});
      ent.push_back({face_cells[2 * f + 1], 1.0});
    });
    s = upload(H, &a->E);
  }
  if (s == FL_OK) {  // Pi = W^-1 |E| (eq. sCF): 1/2 at both cells
    HostEll H = build_ell(F, [&](int64_t f, auto &ent) {
      ent.push_back({face_cells[2 * f], 0.5});
      ent.push_back({face_cells[2 * f + 1], 0.5});
    });
    s = upload(H, &a->Pi);
  }
  // T = 1/2 N (I (x) A) N^T E and -S = -1/2 N (I (x) D^A) N^T E: for every
  // face j sharing a cell c with f (A_fj counts the shared cells, D^A_fj
  // sums E[f, c] over them), (n_f . n_j) / 2 times row j of E
  if (s == FL_OK) {
    HostEll H = build_ell(F, [&](int64_t f, auto &ent) {
      for (int side = 0; side < 2; ++side) {
        const int32_t c = face_cells[2 * f + side];
        for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
          const int32_t j = cf[q];
          if (j == f) continue;
          const double w = 0.5 * dotn(f, j);
          ent.push_back({face_cells[2 * j], -w});
          ent.push_back({face_cells[2 * j + 1], w});
        }
      }
    });
    s = upload(H, &a->T);
  }
  if (s == FL_OK) {
    HostEll H = build_ell(F, [&](int64_t f, auto &ent) {
      for (int side = 0; side < 2; ++side) {
        const int32_t c = face_cells[2 * f + side];
        const double efc = side == 0 ? -1.0 : 1.0;
        for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
          const int32_t j = cf[q];
          if (j == f) continue;
          const double w = -0.5 * efc * dotn(f, j);  // the stored matrix is -S
          ent.push_back({face_cells[2 * j], -w});
          ent.push_back({face_cells[2 * j + 1], w});
        }
      }
    });
    s = upload(H, &a->mS);
  }
  if (s == FL_OK) {  // M = V^-1 E^T diag(A): R_c = sum_f E[f, c] A_f / V_c phi_f
    HostEll H = build_ell(C, [&](int64_t c, auto &ent) {
      for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
        const int32_t f = cf[q];
        const double efc = (face_cells[2 * f] == c) ? -1.0 : 1.0;
        ent.push_back({f, efc * areas[f] / volumes[c]});
      }
    });
    s = upload(H, &a->M);
  }
  if (s != FL_OK) {
    fl_alg_destroy(a);
    return s;
  }
  *out = a;
  return FL_OK;
}

fl_status fl_alg_destroy(fl_alg *a) {
  if (a == nullptr) return FL_OK;
  for (fl_ell *m : {&a->E, &a->Pi, &a->T, &a->mS, &a->M}) free_ell(*m);
  delete a;
  return FL_OK;
}

fl_status fl_alg_info(const fl_alg *a, int64_t *nnz, int32_t *width, size_t *bytes) {
  if (a == nullptr) return fail(FL_EINVAL, "NULL handle");
  const fl_ell *m[5] = {&a->E, &a->T, &a->mS, &a->Pi, &a->M};
  size_t b = 0;
  for (int i = 0; i < 5; ++i) {
    if (nnz) nnz[i] = m[i]->nnz;
    if (width) width[i] = m[i]->width;
    b += ell_bytes(*m[i]);
  }
  if (bytes) *bytes = b;
  return FL_OK;
}

}  // extern "C"

namespace {
// d, r, t_f (|F| each) and R (|C|)
size_t alg_ws_bytes(const fl_alg *a) {
  return 3 * align256((size_t)a->F * 8) + align256((size_t)a->C * 8);
}
}  // namespace

extern "C" {

fl_status fl_alg_workspace_size(const fl_alg *a, size_t *bytes) {
  if (a == nullptr || bytes == nullptr) return fail(FL_EINVAL, "NULL argument");
  *bytes = alg_ws_bytes(a);
  return FL_OK;
}

fl_status fl_alg_face_values(const fl_alg *a, fl_limiter lim, const void *theta, const void *u_f,
                             void *theta_f, void *ws, size_t ws_bytes, void *stream) {
  if (a == nullptr) return fail(FL_EINVAL, "NULL handle");
  fl_status s = check_enums(lim, FL_F64);
  if (s != FL_OK) return s;
  const size_t need = alg_ws_bytes(a);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if ((s = check_buffer(theta, a->C * 8, "theta")) != FL_OK) return s;
  if ((s = check_buffer(u_f, a->F * 8, "u_f")) != FL_OK) return s;
  if ((s = check_buffer(theta_f, a->F * 8, "theta_f")) != FL_OK) return s;
  if ((s = check_buffer(ws, need, "workspace")) != FL_OK) return s;
  if (a->F == 0) return FL_OK;
  char *w = static_cast<char *>(ws);
  double *d = reinterpret_cast<double *>(w);
  double *r = reinterpret_cast<double *>(w + align256((size_t)a->F * 8));
  const cudaError_t e = face_values(a, lim, static_cast<const double *>(theta),
                                    static_cast<const double *>(u_f), d, r,
                                    static_cast<double *>(theta_f), as_stream(stream));
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "algebraic face values");
}

fl_status fl_alg_step_euler(const fl_alg *a, fl_limiter lim, double dt, int64_t nsteps,
                            void *theta, const void *u_f, void *ws, size_t ws_bytes,
                            void *stream) {
  if (a == nullptr) return fail(FL_EINVAL, "NULL handle");
  fl_status s = check_enums(lim, FL_F64);
  if (s != FL_OK) return s;
  if (nsteps < 0) return fail(FL_EINVAL, "nsteps < 0");
  if (!std::isfinite(dt)) return fail(FL_EINVAL, "dt is not finite");
  const size_t need = alg_ws_bytes(a);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if ((s = check_buffer(theta, a->C * 8, "theta")) != FL_OK) return s;
  if ((s = check_buffer(u_f, a->F * 8, "u_f")) != FL_OK) return s;
  if ((s = check_buffer(ws, need, "workspace")) != FL_OK) return s;
  char *w = static_cast<char *>(ws);
  const size_t fb = align256((size_t)a->F * 8);
  double *d = reinterpret_cast<double *>(w);
  double *r = reinterpret_cast<double *>(w + fb);
  double *t = reinterpret_cast<double *>(w + 2 * fb);
  double *R = reinterpret_cast<double *>(w + 3 * fb);
  double *th = static_cast<double *>(theta);
  const double *u = static_cast<const double *>(u_f);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaSuccess;
  for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
    // Algorithm 5: theta <- theta + dt M U(u_f) theta_f
    e = face_values(a, lim, th, u, d, r, t, st);
    if (e == cudaSuccess) {
      k_uxty<<<grid_for(a->F), AT, 0, st>>>(u, t, d, a->F);  // phi into d
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spmv(a->M, d, R, false, st);
    if (e == cudaSuccess) {
      k_axpy<<<grid_for(a->C), AT, 0, st>>>(dt, R, th, a->C);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "algebraic Euler step");
}

}  // extern "C"
