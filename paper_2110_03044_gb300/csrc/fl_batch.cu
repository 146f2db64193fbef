// fl_batch.cu -- many independent periodic boxes advanced together: one
// persistent launch per RK stage over a single work list of (box, tile)
// items, replayed from a captured CUDA graph.
//
// Every box keeps its own fields, velocity, spacings and step size; a tile
// is the same 32 x 8 x zchunk column the single-mesh kernel processes.  The
// CTAs of the persistent kernel (as many as fit on the GPU at once) take
// tiles from a shared counter, so boxes of uneven sizes (32^3 .. 128^3)
// balance across the SMs without one launch per box.  The stage parameters
// of every box live in device memory owned by the batch, so one captured
// graph per (limiter, dtype, RK order, z chunk) serves every call; a call
// only refreshes the parameter table (one host-to-device copy) and replays.
//
// The work decomposition is picked by an autotuner on the first call for a
// (limiter, dtype, RK order): each candidate times a few stage-1 launches
// (which write only workspace, never the caller's fields) and the fastest is
// kept.  Candidates:
//   * 32 x 8 rectangles (the single-mesh stage tile, shared memory, one cell
//     per thread) with a z chunk of 8, 16, 32 or 64 planes (FP64 and FP32);
//   * FP32 only: runs of the flat plane (fl_struct_flat.cuh, registers and
//     warp shuffles, no barriers) with 1, 2 or 4 cells per thread 32 cells
//     apart, 4 or 8 warps per CTA and a z chunk of 16, 32 or 64 planes;
//   * FP32 only: runs over padded copies of the boxes (fl_struct_pad4.cuh:
//     periodic ghost cells, 4 consecutive 16-byte aligned cells per thread,
//     loads staged a plane ahead with cp.async), 1, 2, 4 or 8 warps per CTA
//     and a z chunk of 16, 32 or 64 planes; the copies in and out run once
//     per call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "fl_internal.h"
#include "fl_kernels.h"
#include "fl_struct_flat.cuh"
#include "fl_struct_pad4.cuh"
#include "fl_struct_tile.cuh"

namespace fl {
fl_status check_buffer(const void *p, size_t bytes, const char *name);
fl_status check_enums(int lim, fl_dtype dt);
}  // namespace fl

struct fl_batch {
  int n = 0;
  int device = 0;
  std::vector<const fl_mesh *> meshes;
  int64_t cells = 0, faces = 0;
  // parameter tables: 3 stages (RK3) or 2 parities (Euler) x n boxes
  void *d_params = nullptr;
  void *h_params = nullptr;  // pinned staging
  size_t params_bytes = 0;
  cudaEvent_t params_done = nullptr;
  // recorded on the caller's stream after every call's last launch; the next
  // call's stream waits on it before touching the parameter table and the
  // work counters, so calls on different streams run one after the other
  cudaEvent_t last_call = nullptr;
  unsigned *d_counters = nullptr;  // one work counter per stage
  // tile lists per z chunk
  std::map<int, std::pair<int2 *, int>> tiles;
  // tuned work decomposition (an encoded fl::Cfg) per (lim, dtype, rk)
  std::map<std::tuple<int, int, int>, int> tuned;
  // graph cache per (lim, dtype, rk, decomposition)
  std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
};

namespace fl {
namespace {

constexpr int BTY = 8;
constexpr int MAXSTAGES = 3;
// rows of the parameter table: the stages, then the boxes' layout copies
constexpr int CONV_ROW = MAXSTAGES;
constexpr int PARAM_ROWS = MAXSTAGES + 1;

// (FP32 boxes run the shared-memory tile here: in this persistent kernel the
// register tile of fl_struct_reg.cuh measured no faster, 1.61 against 1.60 ms
// for the 64-box SSP-RK3 step, both with 32-bit addressing)
template <class T, int LIM, int SEED, bool PRE>
__global__ void __launch_bounds__(TX *BTY, 4)
    k_batch_stage(const SParams<T> *__restrict__ params, const int2 *__restrict__ tiles,
                  int n_tiles, unsigned *counter) {
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0) s_next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    if (t >= n_tiles) break;
    const int2 bt = tiles[t];
    const SParams<T> p = params[bt.x];
    stage_tile<T, LIM, SEED, BTY, PRE>(p, bt.y);
  }
}

// FP32: items are (box, run + runs-per-plane x z chunk) of the flat tile.
// FL_FLAT_MINB: CTAs of 256 threads the register budget must allow per SM.
// 4 caps the tile at 64 registers without spills (74 uncapped): 8 CTAs of 4
// warps per SM instead of 6, and the 64-box van Leer step ran 1.18 ms
// against 1.50 (5: 48 registers with spills, 1.26 ms).
#ifndef FL_FLAT_MINB
#define FL_FLAT_MINB 4
#endif
template <int LIM, int SEED, int CX>
__global__ void __launch_bounds__(256, FL_FLAT_MINB)
    k_batch_flat(const SParams<float> *__restrict__ params, const int2 *__restrict__ items,
                 int n_items, unsigned *counter) {
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0) s_next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    if (t >= n_items) break;
    const int2 bt = items[t];
    const SParams<float> p = params[bt.x];
    stage_flat<LIM, SEED, CX>(p, bt.y % p.tiles_x, bt.y / p.tiles_x);
  }
}

// FP32 on padded box copies (fl_struct_pad4.cuh): items are (box, run of
// 128 w cells of a plane's rows + runs-per-plane x z chunk); boxes with
// nx < 8 (or a padded copy of 2^31 cells or more) keep their own layout and
// take the one-cell flat tile over runs of 32 w cells.
// FL_PAD4_MAXREG: register cap of the tile (128: 16 warps per SM).
#ifndef FL_PAD4_MAXREG
#define FL_PAD4_MAXREG 128
#endif
template <int LIM, int SEED>
__global__ void __maxnreg__(FL_PAD4_MAXREG)
    k_batch_pad4(const SParams<float> *__restrict__ params, const int2 *__restrict__ items,
                 int n_items, unsigned *counter) {
  __shared__ int s_next;
  extern __shared__ float4 pad_stage[];  // PAD_STAGE_BYTES per thread
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0) s_next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    if (t >= n_items) break;
    const int2 bt = items[t];
    const SParams<float> p = params[bt.x];
    if (p.pitch > 0)
      stage_pad4<LIM, SEED>(p, bt.y % p.tiles_x, bt.y / p.tiles_x,
                            pad_stage + (threadIdx.y * blockDim.x + threadIdx.x) * PAD_STRIDE);
    else stage_flat<LIM, SEED, 1>(p, bt.y % p.tiles_x, bt.y / p.tiles_x);
  }
}

// A work decomposition: kind 0 = 32 x 8 rectangles (z chunk zc), kind 1 =
// flat runs of 32 cx w cells (FP32), kind 2 = runs of 128 w cells of the
// boxes' padded copies, four consecutive cells per thread (FP32), packed
// into one int for the maps.
struct Cfg {
  int kind, cx, w, zc;
};
int encode(const Cfg &c) { return c.zc | (c.kind << 8) | (c.cx << 12) | (c.w << 16); }
Cfg decode(int v) { return Cfg{(v >> 8) & 0xF, (v >> 12) & 0xF, (v >> 16) & 0xFF, v & 0xFF}; }

template <int SEED>
void *flat_kernel(int lim, int cx) {
#define FL_FLAT(L)                                                        \
  case L:                                                                 \
    return cx == 1 ? (void *)k_batch_flat<L, SEED, 1>                     \
                   : cx == 2 ? (void *)k_batch_flat<L, SEED, 2>           \
                             : (void *)k_batch_flat<L, SEED, 4>;
  switch (lim) {
    FL_FLAT(LIM_UPWIND)
    FL_FLAT(LIM_CENTRAL)
    FL_FLAT(LIM_MINMOD)
    FL_FLAT(LIM_VANLEER)
    FL_FLAT(LIM_SUPERBEE)
    FL_FLAT(LIM_SMART)
  }
#undef FL_FLAT
  return nullptr;
}

template <int SEED>
void *pad4_kernel(int lim) {
  switch (lim) {
    case LIM_UPWIND: return (void *)k_batch_pad4<LIM_UPWIND, SEED>;
    case LIM_CENTRAL: return (void *)k_batch_pad4<LIM_CENTRAL, SEED>;
    case LIM_MINMOD: return (void *)k_batch_pad4<LIM_MINMOD, SEED>;
    case LIM_VANLEER: return (void *)k_batch_pad4<LIM_VANLEER, SEED>;
    case LIM_SUPERBEE: return (void *)k_batch_pad4<LIM_SUPERBEE, SEED>;
    case LIM_SMART: return (void *)k_batch_pad4<LIM_SMART, SEED>;
  }
  return nullptr;
}

template <class T, int SEED, bool PRE>
void *kernel_ptr(int lim) {
  switch (lim) {
    case LIM_UPWIND: return (void *)k_batch_stage<T, LIM_UPWIND, SEED, PRE>;
    case LIM_CENTRAL: return (void *)k_batch_stage<T, LIM_CENTRAL, SEED, PRE>;
    case LIM_MINMOD: return (void *)k_batch_stage<T, LIM_MINMOD, SEED, PRE>;
    case LIM_VANLEER: return (void *)k_batch_stage<T, LIM_VANLEER, SEED, PRE>;
    case LIM_SUPERBEE: return (void *)k_batch_stage<T, LIM_SUPERBEE, SEED, PRE>;
    case LIM_SMART: return (void *)k_batch_stage<T, LIM_SMART, SEED, PRE>;
  }
  return nullptr;
}

// pre: FP64 boxes fold the flux product into the cell update with the
// pre-scaled velocity w = dt (A/V) u of every box (as fl_step_rk does)
void *batch_kernel(fl_dtype dt, int lim, int seed, bool pre, int cfg) {
  const Cfg c = decode(cfg);
  if (dt == FL_F32 && c.kind == 1)
    return seed == SEED_PLAIN ? flat_kernel<SEED_PLAIN>(lim, c.cx)
                              : flat_kernel<SEED_COMBINE>(lim, c.cx);
  if (dt == FL_F32 && c.kind == 2)
    return seed == SEED_PLAIN ? pad4_kernel<SEED_PLAIN>(lim) : pad4_kernel<SEED_COMBINE>(lim);
  if (dt == FL_F64) {
    if (pre)
      return seed == SEED_PLAIN ? kernel_ptr<double, SEED_PLAIN, true>(lim)
                                : kernel_ptr<double, SEED_COMBINE, true>(lim);
    return seed == SEED_PLAIN ? kernel_ptr<double, SEED_PLAIN, false>(lim)
                              : kernel_ptr<double, SEED_COMBINE, false>(lim);
  }
  return seed == SEED_PLAIN ? kernel_ptr<float, SEED_PLAIN, false>(lim)
                            : kernel_ptr<float, SEED_COMBINE, false>(lim);
}

bool batch_prescales(fl_dtype dt) { return dt == FL_F64; }

// boxes a kind-2 decomposition copies into the padded layout (the tile's
// offsets are 32-bit: a copy of 2^31 cells or more stays in the box's layout)
bool box_padded(const fl_mesh *m) {
  return m->nx >= 8 && pad_geom(m->nx, m->ny, m->nz).vol < (1LL << 31);
}

// work items of a box: rectangles (kind 0) or flat runs (kinds 1, 2) per plane
int tiles_x_of(const fl_mesh *m, const Cfg &c) {
  if (c.kind == 2 && box_padded(m)) {
    const long long run = 128LL * c.w;
    return (int)(((long long)pad_geom(m->nx, m->ny, m->nz).P * m->ny + run - 1) / run);
  }
  if (c.kind != 0) {
    const long long run = 32LL * c.cx * c.w;
    return (int)(((long long)m->nx * m->ny + run - 1) / run);
  }
  return (m->nx + TX - 1) / TX;
}
int tiles_y_of(const fl_mesh *m, const Cfg &c) {
  return c.kind != 0 ? 1 : (m->ny + BTY - 1) / BTY;
}
int zchunk_of(const fl_mesh *m, int zc) { return std::min(zc, m->nz); }

// (box, item) list of a decomposition; items of one box are contiguous
fl_status get_tiles(fl_batch *b, int cfg, int2 **d, int *n) {
  auto it = b->tiles.find(cfg);
  if (it != b->tiles.end()) {
    *d = it->second.first;
    *n = it->second.second;
    return FL_OK;
  }
  const Cfg c = decode(cfg);
  std::vector<int2> h;
  for (int i = 0; i < b->n; ++i) {
    const fl_mesh *m = b->meshes[i];
    const int z = zchunk_of(m, c.zc);
    const long long nt = (long long)tiles_x_of(m, c) * tiles_y_of(m, c) * ((m->nz + z - 1) / z);
    for (long long t = 0; t < nt; ++t) h.push_back(make_int2(i, (int)t));
  }
  if (h.size() >= (1u << 31)) return fail(FL_EUNSUPPORTED, "too many tiles");
  int2 *dp = nullptr;
  if (cudaMalloc(&dp, h.size() * sizeof(int2)) != cudaSuccess)
    return fail(FL_ENOMEM, "tile list allocation failed");
  if (cudaMemcpy(dp, h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dp);
    return fail(FL_ECUDA, "tile list upload failed");
  }
  b->tiles[cfg] = {dp, (int)h.size()};
  *d = dp;
  *n = (int)h.size();
  return FL_OK;
}

template <class T>
SParams<T> box_params(const fl_mesh *m, int cfg, const void *x, const void *thn, void *y,
                      const void *u, double dtime, int seed, double a, double bcoef) {
  const Cfg c = decode(cfg);
  SParams<T> p;
  p.x = static_cast<const T *>(x);
  p.thn = static_cast<const T *>(thn);
  p.y = static_cast<T *>(y);
  p.thf = nullptr;
  p.u = static_cast<const T *>(u);
  p.nx = m->nx;
  p.ny = m->ny;
  p.nz = m->nz;
  p.act_x = m->act[0];
  p.act_y = m->act[1];
  p.act_z = m->act[2];
  p.ux_off = m->u_off[0];
  p.uy_off = m->u_off[1];
  p.uz_off = m->u_off[2];
  p.plane = (long long)m->nx * m->ny;
  const double sc = (seed == SEED_PLAIN) ? dtime : bcoef * dtime;
  p.cx = (T)(sc / m->hx);
  p.cy = (T)(sc / m->hy);
  p.cz = (T)(sc / m->hz);
  p.a = blend_a<T>(a, bcoef);
  p.b = (T)bcoef;
  p.g = (T)1;
  p.flip = 0;
  p.codes = nullptr;
  p.tiles_x = tiles_x_of(m, c);
  p.tiles_y = tiles_y_of(m, c);
  p.zchunk = zchunk_of(m, c.zc);
  return p;
}

size_t param_size(fl_dtype dt) { return dt == FL_F64 ? sizeof(SParams<double>) : sizeof(SParams<float>); }

// Padded copy of box i for a kind-2 decomposition: theta, the RK stage
// buffers, then the active velocity components, each block 256-byte aligned.
size_t pad_block(const fl_mesh *m) {
  return align256((size_t)pad_geom(m->nx, m->ny, m->nz).vol * sizeof(float));
}
size_t pad_bytes(const fl_mesh *m, int rk) {
  const int na = m->act[0] + m->act[1] + m->act[2];
  return (rk == 3 ? 3 : 2) * pad_block(m) +
         align256((size_t)na * pad_geom(m->nx, m->ny, m->nz).vol * sizeof(float));
}

// Workspace of box i: its RK stage buffers, then (pre) its w_f; for FP32 at
// least the padded copy of a kind-2 decomposition (both start at the box's
// offset, one decomposition being in use at a time).
size_t box_ws_bytes(const fl_mesh *m, fl_dtype dt, int rk) {
  size_t t = (rk == 3 ? 2 : 1) * align256((size_t)m->C * dsize(dt));
  if (batch_prescales(dt)) t += align256((size_t)m->F * dsize(dt));
  if (dt == FL_F32 && box_padded(m)) t = std::max(t, pad_bytes(m, rk));
  return t;
}

// Stage parameters p of box m moved onto its padded copy at base (theta,
// RK stage buffers A and B, velocities): x, thn and y are picked by the
// caller from those blocks.
void pad_params(SParams<float> &p, const fl_mesh *m, const char *ubase) {
  const PadGeom g = pad_geom(m->nx, m->ny, m->nz);
  p.pitch = g.P;
  p.gy = g.gy;
  p.gz = g.gz;
  p.plane = g.plane;
  p.u = reinterpret_cast<const float *>(ubase);
  p.ux_off = m->u_off[0] / m->C * g.vol;
  p.uy_off = m->u_off[1] / m->C * g.vol;
  p.uz_off = m->u_off[2] / m->C * g.vol;
}

// Fill the staging table: stage s of box i at index s * n + i.  With pre,
// every stage reads the box's w_f (left in its workspace by prescale_boxes).
template <class T>
void fill_params(fl_batch *b, int rk, int cfg, const double *dtv, void *const *theta,
                 const void *const *u, char *ws, size_t es, bool pre) {
  SParams<T> *h = static_cast<SParams<T> *>(b->h_params);
  const bool padded = decode(cfg).kind == 2;
  size_t off = 0;
  for (int i = 0; i < b->n; ++i) {
    const fl_mesh *m = b->meshes[i];
    const size_t one = align256((size_t)m->C * es);
    void *A = ws + off;
    void *B = ws + off + one;
    const void *uw = pre ? static_cast<const void *>(ws + off + (rk == 3 ? 2 : 1) * one) : u[i];
    // the box's layout copy (a kind-2 decomposition of a box with nx >= 8)
    SParams<T> &conv = h[CONV_ROW * b->n + i];
    conv = SParams<T>();
    if constexpr (sizeof(T) == 4) {
      if (padded && box_padded(m)) {
        const size_t V = pad_block(m);
        char *tp = ws + off, *ap = ws + off + V, *bp = ws + off + 2 * V;
        char *up = ws + off + (rk == 3 ? 3 : 2) * V;
        conv = box_params<T>(m, cfg, theta[i], ap, tp, u[i], dtv[i], SEED_PLAIN, 0.0, 1.0);
        conv.thf = reinterpret_cast<T *>(up);
        conv.pitch = pad_geom(m->nx, m->ny, m->nz).P;
        auto st = [&](const char *x, const char *thn, char *y, int seed, double a, double bc) {
          SParams<T> q = box_params<T>(m, cfg, x, thn, y, u[i], dtv[i], seed, a, bc);
          pad_params(q, m, up);
          return q;
        };
        if (rk == 3) {
          h[0 * b->n + i] = st(tp, tp, ap, SEED_PLAIN, 0.0, 1.0);
          h[1 * b->n + i] = st(ap, tp, bp, SEED_COMBINE, 0.75, 0.25);
          h[2 * b->n + i] = st(bp, tp, tp, SEED_COMBINE, 1.0 / 3.0, 2.0 / 3.0);
        } else {
          h[0 * b->n + i] = st(tp, tp, ap, SEED_PLAIN, 0.0, 1.0);
          h[1 * b->n + i] = st(ap, ap, tp, SEED_PLAIN, 0.0, 1.0);
        }
        off += box_ws_bytes(m, FL_F32, rk);
        continue;
      }
    }
    off += box_ws_bytes(m, es == 8 ? FL_F64 : FL_F32, rk);
    if (rk == 3) {
      h[0 * b->n + i] = box_params<T>(m, cfg, theta[i], theta[i], A, uw, dtv[i], SEED_PLAIN, 0.0, 1.0);
      h[1 * b->n + i] = box_params<T>(m, cfg, A, theta[i], B, uw, dtv[i], SEED_COMBINE, 0.75, 0.25);
      h[2 * b->n + i] =
          box_params<T>(m, cfg, B, theta[i], theta[i], uw, dtv[i], SEED_COMBINE, 1.0 / 3.0, 2.0 / 3.0);
    } else {  // Euler: even step theta -> A, odd step A -> theta
      h[0 * b->n + i] = box_params<T>(m, cfg, theta[i], theta[i], A, uw, dtv[i], SEED_PLAIN, 0.0, 1.0);
      h[1 * b->n + i] = box_params<T>(m, cfg, A, A, theta[i], uw, dtv[i], SEED_PLAIN, 0.0, 1.0);
    }
  }
}

size_t batch_ws_bytes(const fl_batch *b, fl_dtype dt, int rk) {
  size_t t = 0;
  for (const fl_mesh *m : b->meshes) t += box_ws_bytes(m, dt, rk);
  return t;
}

// w_f = dt_i (A/V) u_f of every box into its workspace (once per call)
cudaError_t prescale_boxes(fl_batch *b, fl_dtype dt, int rk, const double *dtv,
                           const void *const *u, char *ws, cudaStream_t st) {
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    const fl_mesh *m = b->meshes[i];
    const size_t one = align256((size_t)m->C * dsize(dt));
    e = struct_scale_faces(m, dt, u[i], ws + off + (rk == 3 ? 2 : 1) * one, dtv[i], st);
    off += box_ws_bytes(m, dt, rk);
  }
  return e;
}

dim3 block_of(int cfg) {
  const Cfg c = decode(cfg);
  return c.kind != 0 ? dim3(32, c.w) : dim3(TX, BTY);
}

// dynamic shared memory of a launch: the staging slots of kind 2
size_t smem_of(fl_dtype dt, int cfg) {
  const Cfg c = decode(cfg);
  return dt == FL_F32 && c.kind == 2 ? (size_t)PAD_STAGE_BYTES * 32 * c.w : 0;
}

// the kernels of a decomposition may take its dynamic shared memory (set
// before any launch or occupancy query, outside graph capture)
cudaError_t allow_smem(fl_dtype dt, int lim, bool pre, int cfg) {
  const size_t smem = smem_of(dt, cfg);
  if (smem <= 48 * 1024) return cudaSuccess;
  for (int seed : {SEED_PLAIN, SEED_COMBINE}) {
    const cudaError_t e = cudaFuncSetAttribute(batch_kernel(dt, lim, seed, pre, cfg),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int persistent_grid(fl_dtype dt, int lim, int seed, bool pre, int cfg) {
  const dim3 b = block_of(cfg);
  return resident_ctas(batch_kernel(dt, lim, seed, pre, cfg), (int)(b.x * b.y), smem_of(dt, cfg));
}

// Enqueue one launch of stage s (seed) on st.
cudaError_t enqueue_stage(fl_batch *b, fl_dtype dt, int lim, int s, int seed, bool pre, int cfg,
                          int2 *tiles, int nt, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_counters + s, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const char *params = static_cast<const char *>(b->d_params) + (size_t)s * b->n * param_size(dt);
  unsigned *ctr = b->d_counters + s;
  void *args[] = {(void *)&params, (void *)&tiles, (void *)&nt, (void *)&ctr};
  return cudaLaunchKernel(batch_kernel(dt, lim, seed, pre, cfg),
                          dim3(persistent_grid(dt, lim, seed, pre, cfg)), block_of(cfg), args,
                          smem_of(dt, cfg), st);
}

// Kind 2: copy theta and the velocities of the padded boxes into their
// padded copies (in), or theta back (out; from the RK stage buffer A when
// alt is set).  One launch over all boxes, blockIdx.y = box.
cudaError_t pad_copy(fl_batch *b, bool in, bool alt, cudaStream_t st) {
  long long most = 1;  // rows of the largest box
  for (const fl_mesh *m : b->meshes)
    if (box_padded(m)) {
      const PadGeom g = pad_geom(m->nx, m->ny, m->nz);
      most = std::max(most, in ? (long long)g.PY * g.PZ : (long long)m->ny * m->nz);
    }
  const int gx = (int)std::min<long long>((most + 7) / 8, 1024);
  const SParams<float> *conv = static_cast<const SParams<float> *>(b->d_params) + CONV_ROW * b->n;
  if (in) k_pad_in<<<dim3(gx, b->n), dim3(32, 8), 0, st>>>(conv);
  else k_pad_out<<<dim3(gx, b->n), dim3(32, 8), 0, st>>>(conv, alt ? 1 : 0);
  return cudaGetLastError();
}

// Stage launches of one step (RK3: 3 stages; Euler: 2 steps, even and odd).
cudaError_t enqueue_step(fl_batch *b, fl_dtype dt, int lim, int rk, bool pre, int cfg,
                         int2 *tiles, int nt, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (rk == 3) {
    e = enqueue_stage(b, dt, lim, 0, SEED_PLAIN, pre, cfg, tiles, nt, st);
    if (e == cudaSuccess) e = enqueue_stage(b, dt, lim, 1, SEED_COMBINE, pre, cfg, tiles, nt, st);
    if (e == cudaSuccess) e = enqueue_stage(b, dt, lim, 2, SEED_COMBINE, pre, cfg, tiles, nt, st);
  } else {
    e = enqueue_stage(b, dt, lim, 0, SEED_PLAIN, pre, cfg, tiles, nt, st);
    if (e == cudaSuccess) e = enqueue_stage(b, dt, lim, 1, SEED_PLAIN, pre, cfg, tiles, nt, st);
  }
  return e;
}

fl_status upload_params(fl_batch *b, fl_dtype dt, int rk, int cfg, const double *dtv,
                        void *const *theta, const void *const *u, void *ws, bool pre,
                        cudaStream_t st) {
  // the staging buffer may still feed the previous call's copy
  if (cudaEventSynchronize(b->params_done) != cudaSuccess) return fail(FL_ECUDA, "event sync");
  if (dt == FL_F64)
    fill_params<double>(b, rk, cfg, dtv, theta, u, static_cast<char *>(ws), 8, pre);
  else
    fill_params<float>(b, rk, cfg, dtv, theta, u, static_cast<char *>(ws), 4, pre);
  const size_t bytes = (size_t)PARAM_ROWS * b->n * param_size(dt);
  cudaError_t e = cudaMemcpyAsync(b->d_params, b->h_params, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->params_done, st);
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "parameter upload");
}

// Autotune the work decomposition with timed stage-1 launches (they write
// workspace only): the candidates of the file header, fastest kept.
fl_status tune(fl_batch *b, fl_dtype dt, int lim, int rk, const double *dtv, void *const *theta,
               const void *const *u, void *ws, bool pre, cudaStream_t st, int *best) {
  std::vector<int> cand;
  for (int zc : {8, 16, 32, 64}) cand.push_back(encode(Cfg{0, 0, BTY, zc}));
  if (dt == FL_F32) {
    for (int cx : {1, 2, 4})
      for (int w : {4, 8})
        for (int zc : {16, 32, 64}) cand.push_back(encode(Cfg{1, cx, w, zc}));
    for (int w : {1, 2, 4, 8})
      for (int zc : {16, 32, 64}) cand.push_back(encode(Cfg{2, 1, w, zc}));
  }
  float best_ms = 1e30f;
  *best = cand[0];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(FL_ECUDA, "autotune event creation failed");
  }
  fl_status s = FL_OK;
  for (int cfg : cand) {
    int2 *tiles;
    int nt;
    if ((s = get_tiles(b, cfg, &tiles, &nt)) != FL_OK) break;
    if ((s = upload_params(b, dt, rk, cfg, dtv, theta, u, ws, pre, st)) != FL_OK) break;
    cudaError_t e = allow_smem(dt, lim, pre, cfg);
    if (e == cudaSuccess && decode(cfg).kind == 2) e = pad_copy(b, true, false, st);
    if (e == cudaSuccess) e = enqueue_stage(b, dt, lim, 0, SEED_PLAIN, pre, cfg, tiles, nt, st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r)
      e = enqueue_stage(b, dt, lim, 0, SEED_PLAIN, pre, cfg, tiles, nt, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune launch");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      *best = cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // namespace
}  // namespace fl

using namespace fl;

extern "C" {

fl_status fl_batch_create(int n, const fl_mesh *const *meshes, fl_batch **out) {
  if (out == nullptr) return fail(FL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || meshes == nullptr) return fail(FL_EINVAL, "need n >= 1 meshes");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(FL_ECUDA, "no CUDA device");
  for (int i = 0; i < n; ++i) {
    if (meshes[i] == nullptr) return fail(FL_EINVAL, "mesh %d is NULL", i);
    if (meshes[i]->kind != 0) return fail(FL_EUNSUPPORTED, "mesh %d is not structured", i);
    if (meshes[i]->device != dev) return fail(FL_EINVAL, "mesh %d lives on another device", i);
  }
  fl_batch *b = new (std::nothrow) fl_batch();
  if (!b) return fail(FL_ENOMEM, "host allocation failed");
  b->n = n;
  b->device = dev;
  b->meshes.assign(meshes, meshes + n);
  for (const fl_mesh *m : b->meshes) {
    b->cells += m->C;
    b->faces += m->F;
  }
  b->params_bytes = (size_t)PARAM_ROWS * n * sizeof(SParams<double>);
  cudaError_t e = cudaMalloc(&b->d_params, b->params_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_params, b->params_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, MAXSTAGES * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->params_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last_call, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fl_batch_destroy(b);
    return fail(FL_ENOMEM, "batch allocation failed");
  }
  *out = b;
  return FL_OK;
}

fl_status fl_batch_workspace_size(const fl_batch *b, fl_dtype dt, int rk, size_t *bytes) {
  if (b == nullptr || bytes == nullptr) return fail(FL_EINVAL, "NULL argument");
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (dt != FL_F32 && dt != FL_F64) return fail(FL_EINVAL, "unknown dtype");
  *bytes = batch_ws_bytes(b, dt, rk);
  return FL_OK;
}

fl_status fl_batch_step_rk(fl_batch *b, fl_limiter lim, fl_dtype dt, int rk, const double *dtv,
                           int64_t nsteps, void *const *theta, const void *const *u_f, void *ws,
                           size_t ws_bytes, void *stream) {
  if (b == nullptr) return fail(FL_EINVAL, "batch is NULL");
  fl_status s = check_enums(lim, dt);
  if (s != FL_OK) return s;
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (nsteps < 0) return fail(FL_EINVAL, "nsteps < 0");
  if (!dtv || !theta || !u_f) return fail(FL_EINVAL, "NULL argument array");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return fail(FL_EINVAL, "batch was created on another device");
  const size_t es = dsize(dt);
  for (int i = 0; i < b->n; ++i) {
    const fl_mesh *m = b->meshes[i];
    if (!std::isfinite(dtv[i])) return fail(FL_EINVAL, "dt[%d] is not finite", i);
    if ((s = check_buffer(theta[i], m->C * es, "theta[i]")) != FL_OK) return s;
    if ((s = check_buffer(u_f[i], m->F * es, "u_f[i]")) != FL_OK) return s;
  }
  const size_t need = batch_ws_bytes(b, dt, rk);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return fail(FL_EINVAL, "workspace must be 256-byte aligned");
  if ((s = check_buffer(ws, need, "workspace")) != FL_OK) return s;
  if (nsteps == 0) return FL_OK;
  cudaStream_t st = as_stream(stream);
  // the previous call's launches (perhaps on another stream) read the
  // parameter table and the work counters this call rewrites: wait for them
  if (cudaStreamWaitEvent(st, b->last_call, 0) != cudaSuccess)
    return fail(FL_ECUDA, "ordering after the previous batched call failed");
  // pre-scaled velocities (FP64) when every dt is positive (keeps signs)
  bool pre = batch_prescales(dt);
  for (int i = 0; i < b->n && pre; ++i) pre = dtv[i] > 0;
  if (pre) {
    const cudaError_t e = prescale_boxes(b, dt, rk, dtv, u_f, static_cast<char *>(ws), st);
    if (e != cudaSuccess) return cuda_fail(e, "velocity pre-scaling");
  }
  // work decomposition: tuned once per (limiter, dtype, rk, pre)
  const auto tkey = std::make_tuple((int)lim, (int)dt * 2 + (pre ? 1 : 0), rk);
  int cfg;
  auto tit = b->tuned.find(tkey);
  if (tit == b->tuned.end()) {
    if ((s = tune(b, dt, lim, rk, dtv, theta, u_f, ws, pre, st, &cfg)) != FL_OK) return s;
    b->tuned[tkey] = cfg;
  } else {
    cfg = tit->second;
  }
  int2 *tiles;
  int nt;
  if ((s = get_tiles(b, cfg, &tiles, &nt)) != FL_OK) return s;
  if ((s = upload_params(b, dt, rk, cfg, dtv, theta, u_f, ws, pre, st)) != FL_OK) return s;
  const bool padded = dt == FL_F32 && decode(cfg).kind == 2;
  {
    cudaError_t e = allow_smem(dt, lim, pre, cfg);
    if (e == cudaSuccess && padded) e = pad_copy(b, true, false, st);
    if (e != cudaSuccess) return cuda_fail(e, "padded copy in");
  }
  // one graph per (limiter, dtype + pre, rk, decomposition): a step's stage launches
  const auto gkey = std::make_tuple((int)lim, (int)dt * 2 + (pre ? 1 : 0), rk, cfg);
  cudaGraphExec_t exec = nullptr;
  auto git = b->graphs.find(gkey);
  if (git != b->graphs.end()) {
    exec = git->second;
  } else {
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      return fail(FL_ECUDA, "stream creation failed");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_step(b, dt, lim, rk, pre, cfg, tiles, nt, cap);
      e = cudaStreamEndCapture(cap, &g);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    b->graphs[gkey] = exec;
  }
  cudaError_t e = cudaSuccess;
  if (rk == 3) {
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) e = cudaGraphLaunch(exec, st);
  } else {
    // a graph is two Euler steps (theta -> A -> theta); an odd tail runs the
    // even stage alone and copies A back
    for (int64_t n = 0; n + 1 < nsteps && e == cudaSuccess; n += 2) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess && (nsteps & 1)) {
      e = enqueue_stage(b, dt, lim, 0, SEED_PLAIN, pre, cfg, tiles, nt, st);
      size_t off = 0;
      for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const fl_mesh *m = b->meshes[i];
        if (!(padded && box_padded(m)))
          e = cudaMemcpyAsync(theta[i], static_cast<char *>(ws) + off, m->C * es,
                              cudaMemcpyDeviceToDevice, st);
        off += box_ws_bytes(m, dt, rk);
      }
    }
  }
  if (padded && e == cudaSuccess) e = pad_copy(b, false, rk == 1 && (nsteps & 1), st);
  if (e == cudaSuccess) e = cudaEventRecord(b->last_call, st);
  if (e != cudaSuccess) return cuda_fail(e, "batched step");
  return FL_OK;
}

fl_status fl_batch_tiling(const fl_batch *b, fl_limiter lim, fl_dtype dt, int rk, int *kind,
                          int *cells_per_thread, int *warps, int *z_chunk) {
  if (b == nullptr) return fail(FL_EINVAL, "batch is NULL");
  fl_status s = check_enums(lim, dt);
  if (s != FL_OK) return s;
  for (int pre : {batch_prescales(dt) ? 1 : 0, batch_prescales(dt) ? 0 : 1}) {
    auto it = b->tuned.find(std::make_tuple((int)lim, (int)dt * 2 + pre, rk));
    if (it == b->tuned.end()) continue;
    const Cfg c = decode(it->second);
    if (kind) *kind = c.kind;
    if (cells_per_thread) *cells_per_thread = c.kind == 1 ? c.cx : c.kind == 2 ? 4 : 1;
    if (warps) *warps = c.w;
    if (z_chunk) *z_chunk = c.zc;
    return FL_OK;
  }
  return fail(FL_EINVAL, "no decomposition chosen yet for this limiter, dtype and rk_order");
}

fl_status fl_batch_set_tiling(fl_batch *b, fl_limiter lim, fl_dtype dt, int rk, int kind,
                              int cells_per_thread, int warps, int z_chunk) {
  if (b == nullptr) return fail(FL_EINVAL, "batch is NULL");
  fl_status s = check_enums(lim, dt);
  if (s != FL_OK) return s;
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (z_chunk < 1 || z_chunk > 255) return fail(FL_EINVAL, "z_chunk must be in 1 .. 255");
  Cfg c{kind, 0, BTY, z_chunk};
  if (kind == 0) {
    if (cells_per_thread != 1 || warps != BTY)
      return fail(FL_EINVAL, "rectangles take 1 cell per thread and %d warps", BTY);
  } else if (kind == 1) {
    if (dt != FL_F32) return fail(FL_EUNSUPPORTED, "flat runs are an FP32 decomposition");
    if (cells_per_thread != 1 && cells_per_thread != 2 && cells_per_thread != 4)
      return fail(FL_EINVAL, "cells_per_thread must be 1, 2 or 4");
    if (warps < 1 || warps > 8) return fail(FL_EINVAL, "warps must be in 1 .. 8");
    c.cx = cells_per_thread;
    c.w = warps;
  } else if (kind == 2) {
    if (dt != FL_F32) return fail(FL_EUNSUPPORTED, "flat runs are an FP32 decomposition");
    if (cells_per_thread != 4) return fail(FL_EINVAL, "kind 2 takes 4 cells per thread");
    if (warps < 1 || warps > 8) return fail(FL_EINVAL, "warps must be in 1 .. 8");
    c.cx = 1;
    c.w = warps;
  } else {
    return fail(FL_EINVAL, "unknown decomposition kind %d", kind);
  }
  for (int pre : {0, 1}) b->tuned[std::make_tuple((int)lim, (int)dt * 2 + pre, rk)] = encode(c);
  return FL_OK;
}

fl_status fl_batch_destroy(fl_batch *b) {
  if (b == nullptr) return FL_OK;
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &kv : b->tiles) cudaFree(kv.second.first);
  if (b->d_params) cudaFree(b->d_params);
  if (b->h_params) cudaFreeHost(b->h_params);
  if (b->d_counters) cudaFree(b->d_counters);
  if (b->params_done) cudaEventDestroy(b->params_done);
  if (b->last_call) cudaEventDestroy(b->last_call);
  delete b;
  return FL_OK;
}

}  // extern "C"
