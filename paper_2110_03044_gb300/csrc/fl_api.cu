// fl_api.cu -- the C ABI (include/fl.h): argument checking, buffer checks,
// dispatch to the kernels, stage sequencing of Euler / SSP-RK3.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <mutex>
#include <utility>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "fl_internal.h"
#include "fl_kernels.h"
#include "fl_unstructured.h"

namespace fl {

namespace {
thread_local char g_msg[512] = "";
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}

fl_status fail(fl_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return st;
}

fl_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return FL_ECUDA;
}

// A device buffer must be device memory of the calling context and hold at
// least `bytes` bytes from p to the end of its allocation, so that no kernel
// of this library can read or write outside what the caller allocated.
typedef CUresult (*addr_range_fn)(CUdeviceptr *, size_t *, CUdeviceptr);

// The driver's allocation-range query, fetched through the runtime so that
// the library has no link-time dependency on the driver library.
addr_range_fn get_addr_range() {
  static addr_range_fn fn = []() -> addr_range_fn {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<addr_range_fn>(f);
  }();
  return fn;
}

typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

bool current_context_id(unsigned long long *id) {
  static ctx_id_fn fn = []() -> ctx_id_fn {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<ctx_id_fn>(f);
  }();
  if (fn == nullptr) return false;
  return fn(nullptr, id) == CUDA_SUCCESS;
}

cudaError_t set_smem_limit(const void *kernel, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, unsigned long long>, int> done;
  unsigned long long ctx = 0;
  if (!current_context_id(&ctx)) {
    // no context yet: bind the current device's primary context, then ask again
    cudaFree(nullptr);
    if (!current_context_id(&ctx))
      return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, ctx);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

fl_status check_buffer(const void *p, size_t bytes, const char *name) {
  if (bytes == 0) return FL_OK;
  if (p == nullptr) return fail(FL_EINVAL, "%s is NULL", name);
  addr_range_fn range = get_addr_range();
  if (range == nullptr) return fail(FL_ECUDA, "CUDA driver entry point unavailable");
  CUdeviceptr base = 0;
  size_t size = 0;
  CUresult r = range(&base, &size, (CUdeviceptr)p);
  if (r == CUDA_ERROR_INVALID_CONTEXT) {
    // no context current on this thread yet: let the runtime bind the
    // primary context of the current device, then ask again
    cudaFree(nullptr);
    r = range(&base, &size, (CUdeviceptr)p);
  }
  if (r != CUDA_SUCCESS)
    return fail(FL_EINVAL, "%s (%p) is not device memory of the current context", name, p);
  const size_t off = (size_t)((CUdeviceptr)p - base);
  if (off + bytes > size)
    return fail(FL_EINVAL, "%s: %zu bytes needed from %p but the allocation ends %zu bytes after it",
                name, bytes, p, size - off);
  return FL_OK;
}

fl_status status_alloc(fl_mesh *m) {
  void *h = nullptr, *d = nullptr;
  if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
    return fail(FL_ENOMEM, "status word allocation failed");
  *static_cast<volatile int *>(h) = 0;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaFreeHost(h);
    return fail(FL_ECUDA, "status word mapping failed");
  }
  m->status_host = static_cast<int *>(h);
  m->status = static_cast<int *>(d);
  return FL_OK;
}

void status_free(fl_mesh *m) {
  if (m->status_host) cudaFreeHost(m->status_host);
  m->status_host = nullptr;
  m->status = nullptr;
}

namespace {
const char *status_name(int s) {
  switch (s) {
    case FL_ETIMEOUT: return "FL_ETIMEOUT (a bounded wait inside a kernel gave up)";
    case FL_EINDEX: return "FL_EINDEX";
    default: return "an error";
  }
}
}  // namespace

// The mesh is usable from the calling thread: it lives on the current device
// and no kernel of an earlier call on it has recorded a device-side error.
// A recorded error is returned once (and cleared) by the first call that
// sees it; that call runs nothing.  A kernel still running when the call
// starts may record its error later: the next call, or fl_mesh_status
// (which synchronises first), reports it.
fl_status check_mesh(const fl_mesh *m) {
  if (m == nullptr) return fail(FL_EINVAL, "mesh is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(FL_ECUDA, "cudaGetDevice failed");
  if (dev != m->device)
    return fail(FL_EINVAL, "mesh was created on device %d but device %d is current", m->device, dev);
  if (m->status_host != nullptr) {
    const int h = __atomic_exchange_n(m->status_host, 0, __ATOMIC_ACQ_REL);
    if (h != 0)
      return fail((fl_status)h,
                  "a kernel launched by an earlier call on this mesh recorded %s; this call "
                  "ran nothing",
                  status_name(h));
  }
  return FL_OK;
}

// the rows [y_begin, y_end) of the planes [z_begin, z_end) of a structured mesh
fl_status check_box(const fl_mesh *m, int y_begin, int y_end, int z_begin, int z_end) {
  if (m->kind != 0) return fail(FL_EUNSUPPORTED, "a plane or row range needs a structured mesh");
  if (z_begin < 0 || z_end < z_begin || z_end > m->nz)
    return fail(FL_EINVAL, "plane range [%d, %d) is not inside [0, %d]", z_begin, z_end, m->nz);
  if (y_begin < 0 || y_end < y_begin || y_end > m->ny)
    return fail(FL_EINVAL, "row range [%d, %d) is not inside [0, %d]", y_begin, y_end, m->ny);
  return FL_OK;
}

// the cell ranges a stage of a local face-based mesh runs on: block-aligned
fl_status check_cell_range(const fl_mesh *m, int64_t c_begin, int64_t c_end) {
  if (m->kind != 1) return fail(FL_EUNSUPPORTED, "a cell range needs a face-based mesh");
  auto ok = [&](int64_t c) { return c == 0 || c == m->n_interior || c == m->n_owned; };
  if (!ok(c_begin) || !ok(c_end) || c_end < c_begin)
    return fail(FL_EINVAL, "cell range [%lld, %lld): each end must be 0, n_interior (%lld) or "
                           "n_owned (%lld)", (long long)c_begin, (long long)c_end,
                (long long)m->n_interior, (long long)m->n_owned);
  return FL_OK;
}

fl_status check_enums(int lim, fl_dtype dt) {
  if (lim < FL_UPWIND || lim > FL_SMART) return fail(FL_EINVAL, "unknown limiter %d", lim);
  if (dt != FL_F32 && dt != FL_F64) return fail(FL_EINVAL, "unknown dtype %d", (int)dt);
  return FL_OK;
}

int resident_ctas(const void *kernel, int threads, size_t smem) {
  static std::mutex mu;
  // one entry per launch shape: a kernel may run with several block sizes
  static std::map<std::tuple<const void *, int, int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(kernel, dev, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  cache[key] = sms * per;
  return sms * per;
}

int pick_zchunk(long long cols, int nz, long long resident, int prologue) {
  if (nz <= 1 || cols <= 0) return nz < 1 ? 1 : nz;
  if (resident < 1) resident = 1;
  long long best_cost = -1;
  int best = nz;
  for (int tz = 1; tz <= nz; ++tz) {
    const int chunk = (nz + tz - 1) / tz;
    if ((nz + chunk - 1) / chunk != tz) continue;  // each distinct chunk length once
    const long long waves = (cols * tz + resident - 1) / resident;
    const long long cost = waves * (chunk + prologue);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = chunk;
    }
  }
  return best;
}

// RK stage buffers only (what fl_step_rk_noalloc needs)
size_t step_stage_bytes(const fl_mesh *m, fl_dtype dt, int rk) {
  const size_t one = align256((size_t)m->C * dsize(dt));
  return rk == 3 ? 2 * one : one;
}

// stage buffers plus, where struct_step uses it, the pre-scaled velocity
size_t step_ws_bytes(const fl_mesh *m, fl_dtype dt, int rk) {
  size_t b = step_stage_bytes(m, dt, rk);
  if (struct_step_prescales(m, dt)) b += align256((size_t)m->F * dsize(dt));
  return b;
}

}  // namespace fl

using namespace fl;

#define FL_TRY(expr)              \
  do {                            \
    fl_status s_ = (expr);        \
    if (s_ != FL_OK) return s_;   \
  } while (0)

extern "C" {

const char *fl_last_error(void) { return fl::g_msg; }

const char *fl_version(void) { return "fl-gb300 0.1 (sm_103a)"; }

fl_status fl_mesh_create_structured(int nx, int ny, int nz, double hx, double hy, double hz,
                                    unsigned periodic_mask, fl_mesh **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(FL_EINVAL, "sizes must be >= 1");
  if (!(hx > 0) || !(hy > 0) || !(hz > 0) || !std::isfinite(hx) || !std::isfinite(hy) ||
      !std::isfinite(hz))
    return fail(FL_EINVAL, "spacings must be finite and > 0");
  const long long C = (long long)nx * ny * nz;
  if (C >= (1LL << 31)) return fail(FL_EUNSUPPORTED, "n_cells must be < 2^31");
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a)
    if (n[a] > 1 && !(periodic_mask & (1u << a)))
      return fail(FL_EUNSUPPORTED, "non-periodic boundaries are not supported (axis %d)", a);
  fl_mesh *m = new (std::nothrow) fl_mesh();
  if (!m) return fail(FL_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return fail(FL_ECUDA, "no CUDA device");
  }
  m->kind = 0;
  m->nx = nx;
  m->ny = ny;
  m->nz = nz;
  m->hx = hx;
  m->hy = hy;
  m->hz = hz;
  m->C = C;
  m->n_owned = m->n_interior = C;
  int na = 0;
  for (int a = 0; a < 3; ++a) {
    m->act[a] = n[a] > 1;
    m->u_off[a] = m->act[a] ? (int64_t)na * C : 0;
    na += m->act[a];
  }
  m->F = (int64_t)na * C;
  if (const fl_status st = status_alloc(m); st != FL_OK) {
    delete m;
    return st;
  }
  *out = m;
  return FL_OK;
}

fl_status fl_mesh_create(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                         const double *face_normals, const double *face_areas,
                         const double *cell_volumes, unsigned flags, fl_mesh **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  return unstruct_create(n_cells, n_faces, face_cells, face_normals, face_areas, cell_volumes,
                         nullptr, flags, n_cells, n_cells, out);
}

fl_status fl_mesh_create_local(int64_t n_cells, int64_t n_owned, int64_t n_interior,
                               int64_t n_faces, const int32_t *face_cells,
                               const double *face_normals, const double *face_areas,
                               const double *cell_volumes, const double *face_distances,
                               unsigned flags, fl_mesh **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_interior < 0 || n_owned < n_interior || n_cells < n_owned)
    return fail(FL_EINVAL, "need 0 <= n_interior <= n_owned <= n_cells");
  return unstruct_create(n_cells, n_faces, face_cells, face_normals, face_areas, cell_volumes,
                         face_distances, flags, n_owned, n_interior, out);
}

fl_status fl_mesh_create_weighted(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                                  const double *face_normals, const double *face_areas,
                                  const double *cell_volumes, const double *face_distances,
                                  unsigned flags, fl_mesh **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_faces > 0 && face_distances == nullptr) return fail(FL_EINVAL, "NULL input array");
  return unstruct_create(n_cells, n_faces, face_cells, face_normals, face_areas, cell_volumes,
                         face_distances, flags, n_cells, n_cells, out);
}

fl_status fl_mesh_permutation(const fl_mesh *m, int32_t *cell_perm, int32_t *face_perm,
                              uint8_t *face_flip) {
  if (m == nullptr) return fail(FL_EINVAL, "mesh is NULL");
  for (int64_t c = 0; cell_perm && c < m->C; ++c)
    cell_perm[c] = m->renumbered ? m->cell_perm[c] : (int32_t)c;
  for (int64_t f = 0; face_perm && f < m->F; ++f)
    face_perm[f] = m->renumbered ? m->face_perm[f] : (int32_t)f;
  for (int64_t f = 0; face_flip && f < m->F; ++f)
    face_flip[f] = m->renumbered ? m->face_flip[f] : 0;
  return FL_OK;
}

fl_status fl_mesh_info(const fl_mesh *m, int64_t *n_cells, int64_t *n_faces, int *kind) {
  if (m == nullptr) return fail(FL_EINVAL, "mesh is NULL");
  if (n_cells) *n_cells = m->C;
  if (n_faces) *n_faces = m->F;
  if (kind) *kind = m->kind;
  return FL_OK;
}

fl_status fl_mesh_status(const fl_mesh *m, void *stream) {
  if (m == nullptr) return fail(FL_EINVAL, "mesh is NULL");
  const cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronisation");
  return check_mesh(m);
}

fl_status fl_mesh_destroy(fl_mesh *m) {
  if (m == nullptr) return FL_OK;
  status_free(m);
  if (m->kind == 1) unstruct_free(m);
  delete m;
  return FL_OK;
}

fl_status fl_conv_limited_apply(const fl_mesh *m, fl_limiter lim, fl_dtype dt, const void *theta_c,
                                const void *u_f, void *rhs_c, void *theta_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(theta_c, m->C * es, "theta_c"));
  FL_TRY(check_buffer(u_f, m->F * es, "u_f"));
  FL_TRY(check_buffer(rhs_c, m->C * es, "rhs_c"));
  if (theta_f) FL_TRY(check_buffer(theta_f, m->F * es, "theta_f"));
  if (m->C == 0) return FL_OK;
  if (m->kind == 1) return unstruct_apply(m, lim, dt, theta_c, u_f, rhs_c, theta_f, as_stream(stream));
  StageArgs s;
  s.x = theta_c;
  s.thn = theta_c;
  s.y = rhs_c;
  s.thf = theta_f;
  s.u = u_f;
  s.seed = 2;
  cudaError_t e = struct_stage(m, lim, dt, s, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "structured apply kernel");
  return FL_OK;
}

fl_status fl_face_selection(const fl_mesh *m, fl_dtype dt, const void *u_f, int32_t *sel,
                            void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(FL_UPWIND, dt));
  FL_TRY(check_buffer(u_f, m->F * dsize(dt), "u_f"));
  FL_TRY(check_buffer(sel, m->F * 16, "sel"));
  if (m->F == 0) return FL_OK;
  cudaError_t e = (m->kind == 1) ? unstruct_selection(m, dt, u_f, sel, as_stream(stream))
                                 : struct_selection(m, dt, u_f, sel, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "selection kernel");
  return FL_OK;
}

fl_status fl_workspace_size(const fl_mesh *m, fl_dtype dt, int rk, size_t *bytes) {
  if (m == nullptr || bytes == nullptr) return fail(FL_EINVAL, "NULL argument");
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (dt != FL_F32 && dt != FL_F64) return fail(FL_EINVAL, "unknown dtype");
  *bytes = step_ws_bytes(m, dt, rk);
  return FL_OK;
}

}  // extern "C"

namespace {

// fl_step_rk and fl_step_rk_modulated: gfac (host, nsteps x stages) or null
fl_status step_rk_impl(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, double dtime,
                       int64_t nsteps, void *theta, const void *u_f, const double *gfac,
                       void *ws, size_t ws_bytes, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (nsteps < 0) return fail(FL_EINVAL, "nsteps < 0");
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(theta, m->C * es, "theta"));
  FL_TRY(check_buffer(u_f, m->F * es, "u_f"));
  const size_t need = step_ws_bytes(m, dt, rk);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return fail(FL_EINVAL, "workspace must be 256-byte aligned");
  FL_TRY(check_buffer(ws, need, "workspace"));
  if (gfac != nullptr) {
    const int64_t ng = nsteps * (rk == 3 ? 3 : 1);
    for (int64_t i = 0; i < ng; ++i)
      if (!std::isfinite(gfac[i])) return fail(FL_EINVAL, "velocity factor %lld is not finite",
                                               (long long)i);
  }
  if (nsteps == 0 || m->C == 0) return FL_OK;
  cudaStream_t st = as_stream(stream);
  if (m->kind == 1) {
    void *W = struct_step_prescales(m, dt) ? static_cast<char *>(ws) + step_stage_bytes(m, dt, rk)
                                           : nullptr;
    return unstruct_step(m, lim, dt, rk, dtime, nsteps, theta, u_f, ws, st, gfac, W);
  }
  if (gfac == nullptr && line_resident_takes(m, dt)) {
    cudaError_t e = line_resident(m, lim, dt, theta, u_f, nsteps, rk, dtime, st);
    if (e != cudaSuccess) return cuda_fail(e, "1D resident kernel");
    return FL_OK;
  }
  char *wsb = static_cast<char *>(ws);
  void *A = wsb;
  void *B = wsb + align256((size_t)m->C * es);
  void *W = struct_step_prescales(m, dt) ? wsb + step_stage_bytes(m, dt, rk) : nullptr;
  const cudaError_t e =
      struct_step(m, lim, dt, rk, dtime, nsteps, theta, u_f, A, B, W, st, gfac);
  if (e != cudaSuccess) return cuda_fail(e, "structured stage kernel");
  return FL_OK;
}

}  // namespace

// One stage over planes [zlo, zhi) of a structured mesh or cells [clo, chi)
// of a local face-based mesh (a negative end: every plane / owned cell): the
// shared body of fl_step_rk_stage, fl_step_rk_stage_planes and
// fl_step_rk_stage_cells.
static fl_status stage_planes(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, int stage,
                              double dtime, int ylo, int yhi, int zlo, int zhi, int64_t clo,
                              int64_t chi, const void *theta_n, const void *x, void *y,
                              const void *u_f, const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (stage < 0 || stage >= (rk == 3 ? 3 : 1))
    return fail(FL_EINVAL, "stage %d does not exist for rk_order %d", stage, rk);
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  const size_t es = dsize(dt), cb = (size_t)m->C * es;
  FL_TRY(check_buffer(x, cb, "x"));
  FL_TRY(check_buffer(y, cb, "y"));
  if (stage > 0) FL_TRY(check_buffer(theta_n, cb, "theta_n"));
  FL_TRY(check_buffer(u_f, (size_t)m->F * es, "u_f"));
  const bool pre = dt == FL_F64 && w_f != nullptr;
  if (pre) {
    if (!(dtime > 0)) return fail(FL_EINVAL, "a pre-scaled velocity needs dt > 0");
    FL_TRY(check_buffer(w_f, (size_t)m->F * es, "w_f"));
  }
  const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
  if (m->C > 0 && xb < yb + cb && yb < xb + cb)
    return fail(FL_EINVAL, "x and y overlap (a stage reads neighbours of x while writing y)");
  if (m->C == 0 || (zhi >= 0 && zhi == zlo) || (yhi >= 0 && yhi == ylo) ||
      (chi >= 0 && chi == clo))
    return FL_OK;
  StageArgs s;
  s.zlo = zlo;
  s.zhi = zhi;
  s.ylo = ylo;
  s.yhi = yhi;
  s.clo = clo;
  s.chi = chi;
  s.x = x;
  s.thn = stage == 0 ? x : theta_n;
  s.y = y;
  s.u = u_f;
  s.w = pre ? w_f : nullptr;
  s.dt = dtime;
  s.seed = stage == 0 ? 0 : 1;
  s.a = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
  s.b = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  const cudaError_t e = (m->kind == 1) ? unstruct_stage(m, lim, dt, s, as_stream(stream))
                                       : struct_stage(m, lim, dt, s, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stage kernel");
  return FL_OK;
}


extern "C" {

fl_status fl_step_rk(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, double dtime,
                     int64_t nsteps, void *theta, const void *u_f, void *ws, size_t ws_bytes,
                     void *stream) {
  return step_rk_impl(m, lim, dt, rk, dtime, nsteps, theta, u_f, nullptr, ws, ws_bytes, stream);
}

fl_status fl_step_rk_modulated(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                               double dtime, int64_t nsteps, void *theta, const void *u_f,
                               const double *g, void *ws, size_t ws_bytes, void *stream) {
  if (g == nullptr && nsteps > 0) return fail(FL_EINVAL, "velocity factors are NULL");
  return step_rk_impl(m, lim, dt, rk, dtime, nsteps, theta, u_f, g, ws, ws_bytes, stream);
}

fl_status fl_step_rk_blocked(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                             double dtime, int64_t nsteps, void *theta, const void *u_f,
                             void *ws, size_t ws_bytes, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  if (m->kind != 0) return fail(FL_EUNSUPPORTED, "temporal blocking needs a structured mesh");
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (nsteps < 0) return fail(FL_EINVAL, "nsteps < 0");
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(theta, m->C * es, "theta"));
  FL_TRY(check_buffer(u_f, m->F * es, "u_f"));
  const size_t need = step_ws_bytes(m, dt, rk);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return fail(FL_EINVAL, "workspace must be 256-byte aligned");
  FL_TRY(check_buffer(ws, need, "workspace"));
  if (nsteps == 0 || m->C == 0) return FL_OK;
  const cudaError_t e =
      struct_step_fused(m, lim, dt, rk, dtime, nsteps, theta, u_f, ws, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "temporally blocked step kernel");
  return FL_OK;
}

fl_status fl_velocity_prescale(const fl_mesh *m, fl_dtype dt, double dtime, const void *u_f,
                               void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(FL_UPWIND, dt));
  if (!(dtime > 0) || !std::isfinite(dtime)) return fail(FL_EINVAL, "dt must be finite and > 0");
  const size_t bytes = (size_t)m->F * dsize(dt);
  FL_TRY(check_buffer(u_f, bytes, "u_f"));
  FL_TRY(check_buffer(w_f, bytes, "w_f"));
  if (m->F == 0) return FL_OK;
  const cudaError_t e = (m->kind == 1)
                            ? unstruct_scale_area(m, dt, u_f, w_f, dtime, as_stream(stream))
                            : struct_scale_faces(m, dt, u_f, w_f, dtime, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "velocity pre-scaling");
  return FL_OK;
}

fl_status fl_step_rk_stage(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, int stage,
                           double dtime, const void *theta_n, const void *x, void *y,
                           const void *u_f, const void *w_f, void *stream) {
  return stage_planes(m, lim, dt, rk, stage, dtime, 0, -1, 0, -1, 0, -1, theta_n, x, y, u_f,
                      w_f, stream);
}

fl_status fl_step_rk_stage_planes(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, int stage,
                                  double dtime, int z_begin, int z_end, const void *theta_n,
                                  const void *x, void *y, const void *u_f, const void *w_f,
                                  void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_box(m, 0, m->ny, z_begin, z_end));
  return stage_planes(m, lim, dt, rk, stage, dtime, 0, -1, z_begin, z_end, 0, -1, theta_n, x, y,
                      u_f, w_f, stream);
}

fl_status fl_step_rk_stage_box(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, int stage,
                               double dtime, int y_begin, int y_end, int z_begin, int z_end,
                               const void *theta_n, const void *x, void *y, const void *u_f,
                               const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_box(m, y_begin, y_end, z_begin, z_end));
  return stage_planes(m, lim, dt, rk, stage, dtime, y_begin, y_end, z_begin, z_end, 0, -1,
                      theta_n, x, y, u_f, w_f, stream);
}

fl_status fl_step_rk_stage_cells(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, int stage,
                                 double dtime, int64_t c_begin, int64_t c_end,
                                 const void *theta_n, const void *x, void *y, const void *u_f,
                                 const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_cell_range(m, c_begin, c_end));
  return stage_planes(m, lim, dt, rk, stage, dtime, 0, -1, 0, -1, c_begin, c_end, theta_n, x, y,
                      u_f, w_f, stream);
}

fl_status fl_mesh_local_info(const fl_mesh *m, int64_t *n_owned, int64_t *n_interior) {
  if (m == nullptr || n_owned == nullptr || n_interior == nullptr)
    return fail(FL_EINVAL, "NULL argument");
  *n_owned = m->n_owned;
  *n_interior = m->n_interior;
  return FL_OK;
}

size_t fl_reduce_workspace_size(void) { return reduce_ws_bytes(); }

fl_status fl_reduce_max_abs(fl_dtype dt, const void *x, int64_t n, double *out, void *ws,
                            void *stream) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  FL_TRY(check_enums(FL_UPWIND, dt));
  if (n < 0) return fail(FL_EINVAL, "n < 0");
  FL_TRY(check_buffer(x, (size_t)n * dsize(dt), "x"));
  FL_TRY(check_buffer(ws, reduce_ws_bytes(), "workspace"));
  int bad = 0;
  cudaError_t e = reduce_max_abs(dt, x, n, ws, as_stream(stream), out, &bad);
  if (e != cudaSuccess) return cuda_fail(e, "reduction");
  if (bad) return fail(FL_ENONFINITE, "non-finite value in input");
  return FL_OK;
}

fl_status fl_reduce_mass(const fl_mesh *m, fl_dtype dt, const void *theta, double *out, void *ws,
                         void *stream) {
  FL_TRY(check_mesh(m));
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  FL_TRY(check_enums(FL_UPWIND, dt));
  FL_TRY(check_buffer(theta, m->C * dsize(dt), "theta"));
  FL_TRY(check_buffer(ws, reduce_ws_bytes(), "workspace"));
  int bad = 0;
  const double *vol = (m->kind == 1) ? unstruct_volumes(m) : nullptr;
  const double vc = m->hx * m->hy * m->hz;
  // the owned cells (all cells but a local mesh's halo)
  cudaError_t e = reduce_mass(dt, theta, vol, vc, m->n_owned, ws, as_stream(stream), out, &bad);
  if (e != cudaSuccess) return cuda_fail(e, "reduction");
  if (bad) return fail(FL_ENONFINITE, "non-finite value in theta");
  return FL_OK;
}

}  // extern "C"
