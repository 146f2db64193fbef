// fl_structured.cu -- fused limited-convection stage on periodic Cartesian
// meshes (Valle et al., Algorithm 4 with the limited reconstruction of
// Algorithm 1; on Cartesian grids the algebraic d_U collapses to Sweby's
// theta_C - theta_U, Section 3.1).
//
// One launch evaluates a whole RK stage: y = a*thn + b*(x + dt R(x)) (or
// R(x) itself for fl_conv_limited_apply).  Each CTA owns a 32 x TY column of
// cells and streams through a chunk of z planes:
//   * theta of the current plane sits in shared memory with a 2-cell halo
//     in x and y (the upstream cell is a second neighbour); the z neighbours
//     of every column live in registers;
//   * every face difference Delta_m = theta_{m+1} - theta_m is computed once
//     and shared: a face needs its own Delta and the upstream one (Delta_{m-1}
//     or Delta_{m+1});
//   * every face flux u_f theta_f is computed once per CTA and reused by the
//     two cells it separates; only the faces on the -x / -y edge of the tile
//     are evaluated by both neighbouring CTAs (same inputs, same code, so the
//     two results are bit-identical and the scheme stays conservative);
//   * theta_f and the fluxes never leave the chip.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"

#include "fl_struct_tile.cuh"
#include "fl_struct_reg.cuh"

namespace fl {

namespace {

// rows of cells per CTA (a tile is 32 x STY); 4 CTAs of 256 threads per SM
#ifndef FL_STRUCT_TY
#define FL_STRUCT_TY 8
#endif
constexpr int STY = FL_STRUCT_TY;

// CTAs per SM of the code-writing variant (run only in the adjoint's
// recomputation): 4 with a few spilled registers measured faster than 3
// without spills (128^3 superbee reverse sweep 121 ms against 133 ms)
#ifndef FL_CODES_MINB
#define FL_CODES_MINB 4
#endif
#ifndef FL_STRUCT_MINB
#define FL_STRUCT_MINB (32 / STY)
#endif
// CTAs per SM of the FP64 van Leer and SMART stages, whose limiter terms
// run on the integer and FP32 pipes (more registers per thread)
#ifndef FL_HEAVY_MINB
#define FL_HEAVY_MINB FL_STRUCT_MINB
#endif
template <class T, int LIM, int SEED, int TY, bool PRE, bool MOD, bool CODES>
__global__ void __launch_bounds__(TX *TY, CODES ? FL_CODES_MINB
                                          : (sizeof(T) == 8 && (LIM == LIM_VANLEER ||
                                                                LIM == LIM_SMART))
                                              ? FL_HEAVY_MINB
                                              : FL_STRUCT_MINB)
    k_struct_stage(const SParams<T> p) {
  stage_tile<T, LIM, SEED, TY, PRE, MOD, CODES>(p, blockIdx.x);
}

// FP32 stage updates: the barrier-free register tile (fl_struct_reg.cuh)
// FP32 stage updates on shapes the TMA kernel does not take run the
// register tile (250^3 superbee SSP-RK3: 0.564 ms per step against 0.684 ms
// for the shared-memory tile)
#ifndef FL_FP32_REG
#define FL_FP32_REG 1
#endif
#ifndef FL_REG_MINB
#define FL_REG_MINB 3
#endif
template <int LIM, int SEED>
__global__ void __launch_bounds__(TX *8, FL_REG_MINB) k_struct_stage_reg(const SParams<float> p) {
  stage_tile_reg<LIM, SEED>(p, blockIdx.x);
}

template <class T, int LIM, int SEED, bool PRE, bool MOD, bool CODES>
cudaError_t launch_stage(const SParams<T> &p0, int tiles_z, cudaStream_t st) {
  constexpr int TY = STY;
  SParams<T> p = p0;
  const dim3 block(TX, TY);
  const long long grid = (long long)p.tiles_x * p.tiles_y * tiles_z;
  if constexpr (FL_FP32_REG && sizeof(T) == 4 && SEED != SEED_APPLY && TY == 8) {
    k_struct_stage_reg<LIM, SEED><<<(unsigned)grid, block, 0, st>>>(p);
  } else {
    k_struct_stage<T, LIM, SEED, TY, PRE, MOD, CODES><<<(unsigned)grid, block, 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <class T, int SEED, bool PRE, bool MOD = false, bool CODES = false>
cudaError_t dispatch_lim(int lim, const SParams<T> &p, int tz, cudaStream_t st) {
  switch (lim) {
    case LIM_UPWIND: return launch_stage<T, LIM_UPWIND, SEED, PRE, MOD, CODES>(p, tz, st);
    case LIM_CENTRAL: return launch_stage<T, LIM_CENTRAL, SEED, PRE, MOD, CODES>(p, tz, st);
    case LIM_MINMOD: return launch_stage<T, LIM_MINMOD, SEED, PRE, MOD, CODES>(p, tz, st);
    case LIM_VANLEER:
      // van Leer's adjoint is linearised from values, not branch codes
      if constexpr (CODES) return cudaErrorInvalidValue;
      else return launch_stage<T, LIM_VANLEER, SEED, PRE, MOD, false>(p, tz, st);
    case LIM_SUPERBEE: return launch_stage<T, LIM_SUPERBEE, SEED, PRE, MOD, CODES>(p, tz, st);
    case LIM_SMART: return launch_stage<T, LIM_SMART, SEED, PRE, MOD, CODES>(p, tz, st);
  }
  return cudaErrorInvalidValue;
}

// w_f = fac_axis u_f for every face block; a product that underflows keeps
// the sign of u_f (smallest subnormal), so the upwind test of w_f equals the
// upwind test of u_f whenever every fac_axis > 0
template <class T>
__global__ void k_scale_faces(const T *u, T *w, long long C, int nblk, T f0, T f1, T f2) {
  using F = FT<T>;
  const long long n = C * nblk;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n;
       f += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(f / C);
    const T c = b == 0 ? f0 : (b == 1 ? f1 : f2);
    const T uf = u[f];
    T v = F::mul(c, uf);
    if (upwind_positive(uf) && !upwind_positive(v)) v = F::val(1);
    w[f] = v;
  }
}

template <class T>
cudaError_t run_stage_t(const fl_mesh *m, int lim, const StageArgs &s, cudaStream_t st) {
  SParams<T> p;
  // pre-scaled velocities: FP64 stage updates (not the bare operator)
  const bool pre = s.w != nullptr && sizeof(T) == 8 && s.seed != SEED_APPLY;
  p.x = static_cast<const T *>(s.x);
  p.thn = static_cast<const T *>(s.thn);
  p.y = static_cast<T *>(s.y);
  p.thf = static_cast<T *>(s.thf);
  p.u = static_cast<const T *>(pre ? s.w : s.u);
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
  // R = sum_axis (A/V) (phi_minus - phi_plus); A/V = 1/h_axis; a velocity
  // factor g scales the fluxes and, when negative, flips every upwind side
  const double g = (s.seed == SEED_APPLY) ? 1.0 : s.g;
  const bool mod = pre && g != 1.0;
  const double sc = (s.seed == SEED_APPLY) ? 1.0 : s.b * s.dt * (pre ? 1.0 : g);
  p.g = (T)g;
  p.flip = (g < 0) ? (sizeof(T) == 8 ? 0x8000000000000000ull : 0x80000000ull) : 0ull;
  p.codes = static_cast<unsigned char *>(s.codes);
  p.cx = (T)(sc / m->hx);
  p.cy = (T)(sc / m->hy);
  p.cz = (T)(sc / m->hz);
  p.a = blend_a<T>(s.a, s.b);
  p.b = (T)s.b;
  p.tiles_x = (m->nx + TX - 1) / TX;
  p.ylo = s.yhi < 0 ? 0 : s.ylo;
  p.yhi = s.yhi < 0 ? m->ny : s.yhi;
  p.tiles_y = (p.yhi - p.ylo + STY - 1) / STY;
  // z chunks: whole waves of co-resident CTAs (the occupancy of the PLAIN
  // kernel stands for all variants: same block, similar registers)
  const long long cols = (long long)p.tiles_x * p.tiles_y;
  const void *kq;
  if constexpr (FL_FP32_REG && sizeof(T) == 4 && STY == 8)
    kq = reinterpret_cast<const void *>(&k_struct_stage_reg<LIM_SUPERBEE, SEED_PLAIN>);
  else
    kq = reinterpret_cast<const void *>(
        &k_struct_stage<T, LIM_SUPERBEE, SEED_PLAIN, STY, false, false, false>);
  const int resident = resident_ctas(kq, TX * STY, 0);
  p.zlo = s.zhi < 0 ? 0 : s.zlo;
  p.zhi = s.zhi < 0 ? m->nz : s.zhi;
  const int nzr = p.zhi - p.zlo;
  const int zchunk = pick_zchunk(cols, nzr, resident, 2);
  p.zchunk = zchunk;
  const int tz = (nzr + zchunk - 1) / zchunk;
  if constexpr (sizeof(T) == 8) {
    if (pre && !mod && s.codes != nullptr) {
      if (s.seed == SEED_PLAIN) return dispatch_lim<T, SEED_PLAIN, true, false, true>(lim, p, tz, st);
      return dispatch_lim<T, SEED_COMBINE, true, false, true>(lim, p, tz, st);
    }
    if (pre && mod) {
      if (s.seed == SEED_PLAIN) return dispatch_lim<T, SEED_PLAIN, true, true>(lim, p, tz, st);
      return dispatch_lim<T, SEED_COMBINE, true, true>(lim, p, tz, st);
    }
    if (pre) {
      if (s.seed == SEED_PLAIN) return dispatch_lim<T, SEED_PLAIN, true>(lim, p, tz, st);
      return dispatch_lim<T, SEED_COMBINE, true>(lim, p, tz, st);
    }
  }
  switch (s.seed) {
    case SEED_PLAIN: return dispatch_lim<T, SEED_PLAIN, false>(lim, p, tz, st);
    case SEED_COMBINE: return dispatch_lim<T, SEED_COMBINE, false>(lim, p, tz, st);
    default: return dispatch_lim<T, SEED_APPLY, false>(lim, p, tz, st);
  }
}

// -------------------------------------------------------------------------
// 1D resident kernel: one CTA keeps a whole periodic line in shared memory
// and runs every step and stage of the rollout in one launch.
template <class T, int LIM>
__global__ void __launch_bounds__(1024) k_line_resident(T *theta, const T *u, int n, int64_t nsteps,
                                                        int rk, T c) {
  using F = FT<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  T *s_x = reinterpret_cast<T *>(smem);  // stage input / output
  T *s_n = s_x + n;                      // theta^n
  T *s_d = s_n + n;                      // Delta_m = x_{m+1} - x_m
  T *s_f = s_d + n;                      // flux of face m+1/2
  T *s_u = s_f + n;
  const int nt = blockDim.x;
  for (int i = threadIdx.x; i < n; i += nt) {
    s_x[i] = theta[i];
    s_u[i] = u[i];
  }
  __syncthreads();
  const int ns = (rk == 3) ? 3 : 1;
  for (int64_t step = 0; step < nsteps; ++step) {
    if (ns == 3)
      for (int i = threadIdx.x; i < n; i += nt) s_n[i] = s_x[i];
    for (int st = 0; st < ns; ++st) {
      for (int i = threadIdx.x; i < n; i += nt) {
        const int ip = (i + 1 == n) ? 0 : i + 1;
        s_d[i] = F::sub(s_x[ip], s_x[i]);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += nt) {
        const int ip = (i + 1 == n) ? 0 : i + 1;
        const int im = (i == 0) ? n - 1 : i - 1;
        const T uf = s_u[i];
        const bool sp = upwind_positive(uf);
        const T thf = limited_face<T, LIM>(sp ? s_x[i] : s_x[ip], s_d[i], sp ? s_d[im] : s_d[ip], sp);
        s_f[i] = face_flux(uf, thf);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += nt) {
        const int im = (i == 0) ? n - 1 : i - 1;
        T acc;
        if (ns == 1 || st == 0) {
          acc = s_x[i];
          acc = F::fma(-c, s_f[i], acc);
          acc = F::fma(c, s_f[im], acc);
        } else {
          // (stage 3: 1 - RN(2/3), so that the two weights sum to exactly 1)
          const T a = (st == 1) ? T(0.75) : T(1) - T(2.0 / 3.0);
          const T b = (st == 1) ? T(0.25) : T(2.0 / 3.0);
          const T cb = (st == 1) ? F::mul(T(0.25), c) : F::mul(T(2.0 / 3.0), c);
          acc = F::fma(a, s_n[i], F::mul(b, s_x[i]));
          acc = F::fma(-cb, s_f[i], acc);
          acc = F::fma(cb, s_f[im], acc);
        }
        s_x[i] = acc;  // every read of s_x in this stage happened before the last barrier
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += nt) theta[i] = s_x[i];
}

// The same rollout spread over a thread-block cluster of LNC CTAs (one SM
// each): GB300's FP64 rate per SM is low (about 1.6 operations per clock),
// so a single CTA is bound by its one SM's FP64 pipe.  CTA r of the cluster
// owns the cells [n r / LNC, n (r+1) / LNC) (at least 2 when n >= 2 LNC) and
// reads the two cells on each side it needs from its neighbours' shared
// memory (distributed shared memory, cluster-mapped addresses).  Stage
// values alternate between two buffers, so one cluster barrier per stage
// orders every neighbour read after the writes it needs and before the
// writes that reuse the buffer.  The per-face and per-cell arithmetic is
// that of k_line_resident, operation for operation, so both give the same
// bits.  Buffers use one stride for all CTAs (LM = ceil(n / LNC) + 4
// entries) so that a neighbour's buffer sits at the same offset.  The
// cluster holds FL_LINE_NC CTAs (16, beyond the portable 8, where the GPU
// can place such a cluster and the line has 2 cells per CTA), else 8.
#ifndef FL_LINE_NC
#define FL_LINE_NC 16
#endif

template <class T, int LIM>
__global__ void __launch_bounds__(1024)
    k_line_cluster(T *theta, const T *u, int n, int64_t nsteps, int rk, T c, int LM) {
  namespace cg = cooperative_groups;
  using F = FT<T>;
  cg::cluster_group cl = cg::this_cluster();
  const int LNC = (int)cl.num_blocks();
  const int r = (int)cl.block_rank();
  const int lo = (int)(((long long)n * r) / LNC);
  const int hi = (int)(((long long)n * (r + 1)) / LNC);
  const int m = hi - lo;  // cells of this CTA; local index j <-> cell lo + j - 2
  const int rl = (r + LNC - 1) % LNC, rr = (r + 1) % LNC;
  const int ml = (int)(((long long)n * (rl + 1)) / LNC) - (int)(((long long)n * rl) / LNC);
  extern __shared__ __align__(16) unsigned char smem[];
  T *buf0 = reinterpret_cast<T *>(smem);  // stage values, two buffers of LM
  T *buf1 = buf0 + LM;
  T *s_n = buf1 + LM;   // theta^n at j
  T *s_d = s_n + LM;    // Delta of local face j (between j and j + 1)
  T *s_f = s_d + LM;    // flux of local face j
  T *s_u = s_f + LM;    // u of local face j
  const int nt = blockDim.x, tid = threadIdx.x;
  // own cells, and the velocities of local faces 1 .. m + 1 (faces of the
  // cells lo - 1 .. hi - 1, the face of cell i lying between i and i + 1)
  for (int j = tid; j < m; j += nt) buf0[j + 2] = theta[lo + j];
  for (int j = tid; j <= m; j += nt) {
    const int cell = (lo + j - 1 + n) % n;
    s_u[j + 1] = u[cell];
  }
  const int ns = (rk == 3) ? 3 : 1;
  T *cur = buf0, *nxt = buf1;
  for (int64_t step = 0; step < nsteps; ++step) {
    for (int st = 0; st < ns; ++st) {
      // every CTA's cur is complete; nobody writes it again before the next barrier
      cl.sync();
      if (ns == 3 && st == 0)
        for (int j = 2 + tid; j < m + 2; j += nt) s_n[j] = cur[j];
      if (tid < 4) {
        if (tid < 2) {
          const T *src = cl.map_shared_rank(cur, (unsigned)rl);
          cur[tid] = src[ml + tid];  // the left neighbour's last two cells
        } else {
          const T *src = cl.map_shared_rank(cur, (unsigned)rr);
          cur[m + tid] = src[tid];   // the right neighbour's first two cells
        }
      }
      __syncthreads();
      for (int j = tid; j < m + 3; j += nt) s_d[j] = F::sub(cur[j + 1], cur[j]);
      __syncthreads();
      for (int j = 1 + tid; j <= m + 1; j += nt) {
        const T uf = s_u[j];
        const bool sp = upwind_positive(uf);
        const T thf = limited_face<T, LIM>(sp ? cur[j] : cur[j + 1], s_d[j],
                                           sp ? s_d[j - 1] : s_d[j + 1], sp);
        s_f[j] = face_flux(uf, thf);
      }
      __syncthreads();
      for (int j = 2 + tid; j < m + 2; j += nt) {
        T acc;
        if (ns == 1 || st == 0) {
          acc = cur[j];
          acc = F::fma(-c, s_f[j], acc);
          acc = F::fma(c, s_f[j - 1], acc);
        } else {
          const T a = (st == 1) ? T(0.75) : T(1) - T(2.0 / 3.0);
          const T b = (st == 1) ? T(0.25) : T(2.0 / 3.0);
          const T cb = (st == 1) ? F::mul(T(0.25), c) : F::mul(T(2.0 / 3.0), c);
          acc = F::fma(a, s_n[j], F::mul(b, cur[j]));
          acc = F::fma(-cb, s_f[j], acc);
          acc = F::fma(cb, s_f[j - 1], acc);
        }
        nxt[j] = acc;
      }
      T *t = cur;
      cur = nxt;
      nxt = t;
    }
  }
  __syncthreads();
  for (int j = tid; j < m; j += nt) theta[lo + j] = cur[j + 2];
  // no CTA leaves while a neighbour may still read its shared memory
  cl.sync();
}

// Launch one cluster of nc CTAs (the cluster size given at launch)
template <class T, int LIM>
cudaError_t launch_line_cluster(int nc, T *th, const T *uu, int n, int64_t nsteps, int rk, T c,
                                cudaStream_t st, bool probe_only, bool *fits) {
  auto k = k_line_cluster<T, LIM>;
  const int LM = (n + nc - 1) / nc + 4;
  const size_t smem = 6 * sizeof(T) * (size_t)LM;
  const int threads = LM >= 1024 ? 1024 : ((LM + 31) / 32) * 32;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nc > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nc, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (probe_only) {
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k, &cfg);
    *fits = e == cudaSuccess && clusters >= 1;
    cudaGetLastError();  // a size the GPU cannot place is an answer, not an error
    return cudaSuccess;
  }
  e = cudaLaunchKernelEx(&cfg, k, th, uu, n, nsteps, rk, c, LM);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <class T>
cudaError_t run_line_cluster_t(int lim, void *theta, const void *u, int n, int64_t nsteps,
                               int rk, double c, cudaStream_t st) {
  T *th = static_cast<T *>(theta);
  const T *uu = static_cast<const T *>(u);
  // the larger cluster where the line gives each CTA 2 cells and the GPU
  // can place it (asked once per device)
  static int big_ok[64] = {0};  // 0 unknown, 1 yes, 2 no
  int dev = 0;
  cudaGetDevice(&dev);
  int nc = 8;
  if (FL_LINE_NC > 8 && n >= 2 * FL_LINE_NC && dev >= 0 && dev < 64) {
    if (big_ok[dev] == 0) {
      bool fits = false;
      launch_line_cluster<T, LIM_UPWIND>(FL_LINE_NC, th, uu, n, nsteps, rk, (T)c, st, true, &fits);
      big_ok[dev] = fits ? 1 : 2;
    }
    if (big_ok[dev] == 1) nc = FL_LINE_NC;
  }
  bool unused = false;
#define FL_LINE_CASE(L)                                                                        \
  case L:                                                                                      \
    return launch_line_cluster<T, L>(nc, th, uu, n, nsteps, rk, (T)c, st, false, &unused);
  switch (lim) {
    FL_LINE_CASE(LIM_UPWIND)
    FL_LINE_CASE(LIM_CENTRAL)
    FL_LINE_CASE(LIM_MINMOD)
    FL_LINE_CASE(LIM_VANLEER)
    FL_LINE_CASE(LIM_SUPERBEE)
    FL_LINE_CASE(LIM_SMART)
  }
#undef FL_LINE_CASE
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t run_line_t(int lim, void *theta, const void *u, int n, int64_t nsteps, int rk, double c,
                       cudaStream_t st) {
  if (n >= 2 * 8) return run_line_cluster_t<T>(lim, theta, u, n, nsteps, rk, c, st);
  const size_t smem = 5 * sizeof(T) * (size_t)n;
  const int threads = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
  T *th = static_cast<T *>(theta);
  const T *uu = static_cast<const T *>(u);
#define FL_LINE_CASE(L)                                                                        \
  case L: {                                                                                    \
    auto k = k_line_resident<T, L>;                                                            \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                         (int)smem);                                           \
    if (e != cudaSuccess) return e;                                                            \
    k<<<1, threads, smem, st>>>(th, uu, n, nsteps, rk, (T)c);                                  \
    return cudaGetLastError();                                                                 \
  }
  switch (lim) {
    FL_LINE_CASE(LIM_UPWIND)
    FL_LINE_CASE(LIM_CENTRAL)
    FL_LINE_CASE(LIM_MINMOD)
    FL_LINE_CASE(LIM_VANLEER)
    FL_LINE_CASE(LIM_SUPERBEE)
    FL_LINE_CASE(LIM_SMART)
  }
#undef FL_LINE_CASE
  return cudaErrorInvalidValue;
}

// -------------------------------------------------------------------------
// Upwind selection dump: (s, C, D, U) per face in the user layout.
template <class T>
__global__ void k_struct_selection(const T *u, int4 *sel, int nx, int ny, int nz, int a0, int a1,
                                   int a2, long long C) {
  const long long nf = C * (a0 + a1 + a2);
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const int blk = (int)(f / C);
    const long long c = f - (long long)blk * C;
    // the blk-th axis of extent > 1
    const int act[3] = {a0, a1, a2};
    int axis = 0;
    for (int q = 0, seen = -1; q < 3; ++q) {
      if (act[q] && ++seen == blk) {
        axis = q;
        break;
      }
    }
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    int d[3] = {0, 0, 0};
    d[axis] = 1;
    auto cell = [&](int di) -> int {
      const int ii = (i + di * d[0] + 4 * nx) % nx;
      const int jj = (j + di * d[1] + 4 * ny) % ny;
      const int kk = (k + di * d[2] + 4 * nz) % nz;
      return ii + nx * (jj + ny * kk);
    };
    const bool sp = upwind_positive(u[f]);
    const int c0 = cell(0), c1 = cell(1);
    int4 o;
    o.x = sp ? 1 : -1;
    o.y = sp ? c0 : c1;
    o.z = sp ? c1 : c0;
    o.w = sp ? cell(-1) : cell(2);
    sel[f] = o;
  }
}

}  // namespace

cudaError_t struct_stage(const fl_mesh *m, int lim, fl_dtype dt, const StageArgs &s, cudaStream_t st) {
  if (dt == FL_F64) return run_stage_t<double>(m, lim, s, st);
  if (struct_tma_eligible(m, s)) {
    const cudaError_t e = struct_stage_tma(m, lim, s, st);
    if (e != cudaErrorNotSupported) return e;
  }
  return run_stage_t<float>(m, lim, s, st);
}

cudaError_t struct_scale_faces(const fl_mesh *m, fl_dtype dt, const void *u, void *w, double fac,
                               cudaStream_t st) {
  double f[3] = {1, 1, 1};
  int nb = 0;
  const double h[3] = {m->hx, m->hy, m->hz};
  for (int a = 0; a < 3; ++a)
    if (m->act[a]) f[nb++] = fac / h[a];
  if (nb == 0 || m->C == 0) return cudaSuccess;
  const long long n = m->C * nb;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  if (dt == FL_F64)
    k_scale_faces<double><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const double *>(u), static_cast<double *>(w), m->C, nb, f[0], f[1], f[2]);
  else
    k_scale_faces<float><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const float *>(u), static_cast<float *>(w), m->C, nb, (float)f[0],
        (float)f[1], (float)f[2]);
  return cudaGetLastError();
}

bool struct_step_prescales(const fl_mesh *m, fl_dtype dt) {
  if (dt != FL_F64) return false;
  if (m->kind == 1) return true;  // face-based meshes: w_f = dt A_f u_f
  return !line_resident_takes(m, dt);
}

cudaError_t struct_step(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                        int64_t nsteps, void *theta, const void *u, void *A, void *B, void *W,
                        cudaStream_t st, const double *gfac) {
  const size_t es = dsize(dt);
  StageArgs s;
  s.u = u;
  s.dt = dtime;
  cudaError_t e = cudaSuccess;
  // FP64 folds the flux product into the cell update with w = dt (A/V) u,
  // computed once per call (dt > 0 keeps the sign of every u_f)
  if (W != nullptr && dtime > 0 && struct_step_prescales(m, dt)) {
    e = struct_scale_faces(m, dt, u, W, dtime, st);
    if (e != cudaSuccess) return e;
    s.w = W;
  }
  if (rk == 1) {
    // Euler: ping-pong between theta and A (a stage reads neighbours of x
    // while writing y, so x and y must differ)
    void *cur = theta, *nxt = A;
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
      s.x = cur;
      s.thn = cur;
      s.y = nxt;
      s.seed = 0;
      s.b = 1.0;
      s.g = gfac ? gfac[n] : 1.0;
      e = struct_stage(m, lim, dt, s, st);
      void *t = cur;
      cur = nxt;
      nxt = t;
    }
    if (e == cudaSuccess && cur != theta)
      e = cudaMemcpyAsync(theta, cur, m->C * es, cudaMemcpyDeviceToDevice, st);
    return e;
  }
  for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
    // th1 = thn + dt R(thn)
    s.x = theta; s.thn = theta; s.y = A; s.seed = 0; s.a = 0.0; s.b = 1.0;
    s.g = gfac ? gfac[3 * n] : 1.0;
    e = struct_stage(m, lim, dt, s, st);
    if (e != cudaSuccess) break;
    // th2 = 3/4 thn + 1/4 (th1 + dt R(th1))
    s.x = A; s.thn = theta; s.y = B; s.seed = 1; s.a = 0.75; s.b = 0.25;
    s.g = gfac ? gfac[3 * n + 1] : 1.0;
    e = struct_stage(m, lim, dt, s, st);
    if (e != cudaSuccess) break;
    // th^{n+1} = 1/3 thn + 2/3 (th2 + dt R(th2)); thn and y are read and
    // written only at the thread's own cell, so y may alias thn
    s.x = B; s.thn = theta; s.y = theta; s.seed = 1; s.a = 1.0 / 3.0; s.b = 2.0 / 3.0;
    s.g = gfac ? gfac[3 * n + 2] : 1.0;
    e = struct_stage(m, lim, dt, s, st);
  }
  return e;
}

size_t line_resident_max_cells(fl_dtype dt) {
  // five arrays in (at most) 200 KiB of shared memory
  return (200u * 1024u) / (5u * dsize(dt));
}

bool line_resident_takes(const fl_mesh *m, fl_dtype dt) {
  return m->kind == 0 && m->nx > 1 && m->ny == 1 && m->nz == 1 &&
         (size_t)m->nx <= line_resident_max_cells(dt);
}

cudaError_t line_resident(const fl_mesh *m, int lim, fl_dtype dt, void *theta, const void *u,
                          int64_t nsteps, int rk, double dtime, cudaStream_t st) {
  if (!line_resident_takes(m, dt)) return cudaErrorInvalidValue;
  const double c = dtime / m->hx;
  return dt == FL_F64 ? run_line_t<double>(lim, theta, u, m->nx, nsteps, rk, c, st)
                      : run_line_t<float>(lim, theta, u, m->nx, nsteps, rk, c, st);
}

cudaError_t struct_selection(const fl_mesh *m, fl_dtype dt, const void *u, int32_t *sel,
                             cudaStream_t st) {
  const long long nf = m->F;
  if (nf == 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (nf + threads - 1) / threads;
  const unsigned g = (unsigned)(blocks > 65535 * 16 ? 65535 * 16 : blocks);
  if (dt == FL_F64)
    k_struct_selection<double><<<g, threads, 0, st>>>(static_cast<const double *>(u),
                                                      reinterpret_cast<int4 *>(sel), m->nx, m->ny,
                                                      m->nz, m->act[0], m->act[1], m->act[2], m->C);
  else
    k_struct_selection<float><<<g, threads, 0, st>>>(static_cast<const float *>(u),
                                                     reinterpret_cast<int4 *>(sel), m->nx, m->ny,
                                                     m->nz, m->act[0], m->act[1], m->act[2], m->C);
  return cudaGetLastError();
}

}  // namespace fl
