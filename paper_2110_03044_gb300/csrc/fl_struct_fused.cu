// fl_struct_fused.cu -- temporally blocked steps on periodic Cartesian
// meshes: the three stages of an SSP-RK3 step, or three forward-Euler steps
// (Algorithm 4), in ONE launch, so that theta^n, u_f and the result cross
// HBM once per launch instead of once per stage.
//
// Method as in fl_structured.cu (Valle et al., Algorithm 4 with the limited
// face values of Algorithm 1; Sweby's stencil on Cartesian grids, Section
// 3.1).  A stage reads its input two cells deep around each output cell
// (the upstream cell is a second neighbour), so an output tile of BX x BY
// cells needs stage 2 on (BX+4) x (BY+4) cells, stage 1 on (BX+8) x (BY+8)
// and theta^n on (BX+12) x (BY+12).  Every CTA recomputes the halo cells it
// needs, from the same inputs with the same code as the CTA that owns them,
// so all copies are bit-identical and the step stays conservative.
//
// A CTA streams through a chunk of z planes as a software pipeline skewed by
// three planes per stage: iteration t evaluates stage 1 on plane z0-4+t,
// stage 2 on plane z0-7+t and stage 3 on plane z0-10+t, each from planes
// that earlier iterations finished.  One barrier separates the face phase
// from the cell phase, a second one the cell phase from the next face phase.
//   * shared memory holds a ring of five planes of each stage's input
//     (theta^n, theta^1, theta^2: the z stencil of plane q is q-2 .. q+2; the
//     theta^n ring has a sixth slot for the plane arriving by cp.async) and
//     the x and y face fluxes of the current plane of each stage;
//   * each thread owns fixed cells of each stage's region and keeps their
//     z-face fluxes in registers (the +z flux of plane q is the -z flux of
//     plane q+1);
//   * every face flux is evaluated once per CTA and used by both its cells;
//   * the theta^n of an RK blend is read from global memory, where the
//     stage-1 loads of a few iterations earlier left it in L2.
// The cost is recomputation: per output cell, stage 1 evaluates 1.88 cells
// and stage 2 1.41 (tile 32 x 16), plus the z-prologue of each chunk.  On
// GB300 that extra arithmetic outweighs the saved HBM traffic (the per-stage
// kernels are bound by instruction issue in FP32 and by the FP64 pipe), so
// fl_step_rk keeps the per-stage kernels; 256^3 superbee SSP-RK3 measured
// 1.03 ms per step here against 0.211 ms (FP32), with 346 MB of DRAM traffic
// per step against 993 MB.
#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"

namespace fl {

namespace {

#ifndef FL_FUSED_F32_NT
#define FL_FUSED_F32_NT 256
#endif
#ifndef FL_FUSED_F32_MINB
#define FL_FUSED_F32_MINB 2
#endif
template <class T>
struct FCfg;
template <>
struct FCfg<float> {
  static constexpr int BX = 32, BY = 16, NT = FL_FUSED_F32_NT, MINB = FL_FUSED_F32_MINB;
};
template <>
struct FCfg<double> {
  static constexpr int BX = 32, BY = 16, NT = 512, MINB = 1;
};

constexpr int NRING = 5;  // planes q-2 .. q+2 of a stage's input
constexpr int NRING0 = 6; // theta^n: the same plus the plane in flight
constexpr int PRO = 10;   // pipeline iterations before the first output plane

template <class T>
struct FParams {
  const T *x;   // theta^n
  T *y;         // result, distinct from x
  const T *ux;  // face velocity block of each active axis (else unused)
  const T *uy;
  const T *uz;
  int nx, ny, nz;
  int ax, ay, az;  // active axes
  int combine;     // stages 2 and 3 blend with theta^n (SSP-RK3)
  T a2, b2, a3, b3;
  T cx[3], cy[3], cz[3];  // per stage: (blend weight) dt / h_axis
  int tiles_x, tiles_y, zchunk;
};

// Shared-memory layout of one precision (in elements of T).  Region s = 0
// is theta^n, s = 1 .. 3 the output of stage s; its cell (i, j) sits at
// index 2 s + i, 2 s + j of the theta^n region.
template <class T>
struct Geo {
  static constexpr int BX = FCfg<T>::BX, BY = FCfg<T>::BY, NT = FCfg<T>::NT;
  __host__ __device__ static constexpr int W(int s) { return BX + 4 * (3 - s); }
  __host__ __device__ static constexpr int H(int s) { return BY + 4 * (3 - s); }
  __host__ __device__ static constexpr int N(int s) { return W(s) * H(s); }
  static constexpr int R0 = 0;
  static constexpr int R1 = R0 + NRING0 * N(0);
  static constexpr int R2 = R1 + NRING * N(1);
  static constexpr int FX1 = R2 + NRING * N(2);
  static constexpr int FY1 = FX1 + H(1) * (W(1) + 1);
  static constexpr int FX2 = FY1 + (H(1) + 1) * W(1);
  static constexpr int FY2 = FX2 + H(2) * (W(2) + 1);
  static constexpr int FX3 = FY2 + (H(2) + 1) * W(2);
  static constexpr int FY3 = FX3 + H(3) * (W(3) + 1);
  static constexpr int END = FY3 + (H(3) + 1) * W(3);
  static constexpr size_t BYTES = END * sizeof(T) + (W(0) + H(0)) * sizeof(int);
};

// asynchronous global -> shared copy of one element (cp.async), completed
// by cp_wait_all; no register staging
template <class T>
__device__ __forceinline__ void cp_async(T *dst, const T *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recent group complete
__device__ __forceinline__ void cp_wait_prev() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__device__ __forceinline__ int wrapn(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Flux u theta_f of the face between t1 (c0) and t2 (c1); t0 lies behind c0
// and t3 behind c1 (the two candidate upstream cells).
template <class T, int LIM>
__device__ __forceinline__ T flux4(T u, T t0, T t1, T t2, T t3) {
  using F = FT<T>;
  const T a = F::sub(t2, t1);
  if constexpr (sizeof(T) == 4) {
    const bool sp = u > 0.0f;
    return native_flux<LIM>(u, sp ? t1 : t2, a, sp ? F::sub(t1, t0) : F::sub(t3, t2));
  } else {
    const bool sp = upwind_positive(u);
    const T b = F::sub(sp ? t1 : t3, sp ? t0 : t2);
    return face_flux(u, limited_face<T, LIM>(sp ? t1 : t2, a, b, sp));
  }
}

// One stage of the pipeline: region sizes, the thread's cells and their
// z-face fluxes.
template <class T, int LIM, int S>
struct Stage {
  using G = Geo<T>;
  using F = FT<T>;
  static constexpr int NT = G::NT;
  static constexpr int W = G::W(S), H = G::H(S), N = W * H;
  static constexpr int WI = G::W(S - 1);  // input region width (2 more per side)
  static constexpr int O = 2 * S;         // theta^n-region index of cell 0
  static constexpr int K = (N + NT - 1) / NT;
  static constexpr int NXF = H * (W + 1), KX = (NXF + NT - 1) / NT;  // x faces of a plane
  static constexpr int NYF = (H + 1) * W, KY = (NYF + NT - 1) / NT;  // y faces of a plane
  T zprev[K], znew[K], thn[K];
  // face velocities of the plane this stage evaluates next, loaded one
  // iteration ahead so that their latency hides behind a whole iteration
  T uxr[KX], uyr[KY], uzr[K];

  // x face f of row j lies between cells f-1 and f (input columns f+1, f+2);
  // y face j of column i between rows j-1 and j (input rows j+1, j+2)
  __device__ __forceinline__ void load_u(const FParams<T> &p, const int *xs, const int *ys,
                                         unsigned zo) {
    const unsigned nx = (unsigned)p.nx;
    if (p.ax) {
#pragma unroll
      for (int k = 0; k < KX; ++k) {
        const int it = threadIdx.x + k * NT;
        if (it < NXF) {
          const int j = it / (W + 1), f = it - j * (W + 1);
          uxr[k] = p.ux[(unsigned)xs[O + f - 1] + (unsigned)ys[O + j] * nx + zo];
        }
      }
    }
    if (p.ay) {
#pragma unroll
      for (int k = 0; k < KY; ++k) {
        const int it = threadIdx.x + k * NT;
        if (it < NYF) {
          const int j = it / W, i = it - j * W;
          uyr[k] = p.uy[(unsigned)xs[O + i] + (unsigned)ys[O + j - 1] * nx + zo];
        }
      }
    }
    if (p.az) load_uz(p, xs, ys, zo, uzr);
  }

  __device__ __forceinline__ static void load_uz(const FParams<T> &p, const int *xs,
                                                 const int *ys, unsigned zo, T (&dst)[K]) {
    const unsigned nx = (unsigned)p.nx;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < N) {
        const int j = e / W, i = e - j * W;
        dst[k] = p.uz[(unsigned)xs[O + i] + (unsigned)ys[O + j] * nx + zo];
      }
    }
  }

  // x and y face fluxes of plane q; in = the input ring's plane q
  __device__ __forceinline__ void xy_faces(const FParams<T> &p, const T *in, T *fx, T *fy) const {
    if (p.ax) {
#pragma unroll
      for (int k = 0; k < KX; ++k) {
        const int it = threadIdx.x + k * NT;
        if (it < NXF) {
          const int j = it / (W + 1), f = it - j * (W + 1);
          const T *r = in + (j + 2) * WI + f;
          fx[it] = flux4<T, LIM>(uxr[k], r[0], r[1], r[2], r[3]);
        }
      }
    }
    if (p.ay) {
#pragma unroll
      for (int k = 0; k < KY; ++k) {
        const int it = threadIdx.x + k * NT;
        if (it < NYF) {
          const int j = it / W, i = it - j * W;
          const T *r = in + j * WI + i + 2;
          fy[it] = flux4<T, LIM>(uyr[k], r[0], r[WI], r[2 * WI], r[3 * WI]);
        }
      }
    }
  }

  // +z face fluxes of plane q of the thread's cells from input planes
  // q-1 .. q+2 with the velocities uz of those faces
  __device__ __forceinline__ static void z_faces(const T *pm1, const T *p0, const T *pp1,
                                                 const T *pp2, const T (&uz)[K], T (&out)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < N) {
        const int j = e / W, i = e - j * W;
        const int o = (j + 2) * WI + i + 2;
        out[k] = flux4<T, LIM>(uz[k], pm1[o], p0[o], pp1[o], pp2[o]);
      }
    }
  }

  // -z faces of the first plane a CTA evaluates (velocities loaded here)
  __device__ __forceinline__ void first_z(const FParams<T> &p, const T *pm2, const T *pm1,
                                          const T *p0, const T *pp1, const int *xs, const int *ys,
                                          unsigned zo_below) {
    T uz[K];
    load_uz(p, xs, ys, zo_below, uz);
    z_faces(pm2, pm1, p0, pp1, uz, zprev);
  }

  // theta^n of the thread's cells on plane q (for the RK blend)
  __device__ __forceinline__ void load_thn(const FParams<T> &p, const int *xs, const int *ys,
                                           unsigned zo) {
    const unsigned nx = (unsigned)p.nx;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < N) {
        const int j = e / W, i = e - j * W;
        thn[k] = p.x[(unsigned)xs[O + i] + (unsigned)ys[O + j] * nx + zo];
      }
    }
  }

  // y = [a thn + b] x + c (phi_minus - phi_plus) summed over the axes, for
  // the thread's cells; x = the input ring's plane q.  Stages before the
  // last write their region's plane (out, W x H); the last stage writes the
  // cells inside the mesh to global memory (gout = y + plane offset).
  __device__ __forceinline__ void update(const FParams<T> &p, bool combine, T a, T b, T cx, T cy,
                                         T cz, const T *in, const T *fx, const T *fy, T *out,
                                         T *gout, int x0, int y0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < N) {
        const int j = e / W, i = e - j * W;
        const T th0 = in[(j + 2) * WI + i + 2];
        T acc = combine ? F::fma(a, thn[k], F::mul(b, th0)) : th0;
        if (p.ax) {
          acc = F::fma(-cx, fx[j * (W + 1) + i + 1], acc);
          acc = F::fma(cx, fx[j * (W + 1) + i], acc);
        }
        if (p.ay) {
          acc = F::fma(-cy, fy[(j + 1) * W + i], acc);
          acc = F::fma(cy, fy[j * W + i], acc);
        }
        if (p.az) {
          acc = F::fma(-cz, znew[k], acc);
          acc = F::fma(cz, zprev[k], acc);
        }
        if (S < 3) {
          out[e] = acc;
        } else if (x0 + i < p.nx && y0 + j < p.ny) {
          gout[(unsigned)(x0 + i) + (unsigned)(y0 + j) * (unsigned)p.nx] = acc;
        }
      }
    }
  }

  __device__ __forceinline__ void rotate() {
#pragma unroll
    for (int k = 0; k < K; ++k) zprev[k] = znew[k];
  }
};

template <class T, int LIM>
__global__ void __launch_bounds__(FCfg<T>::NT, FCfg<T>::MINB)
    k_struct_rk3_fused(const FParams<T> p) {
  using G = Geo<T>;
  constexpr int NT = G::NT;
  constexpr int N0 = G::N(0), N1 = G::N(1), N2 = G::N(2);
  extern __shared__ __align__(16) unsigned char smem[];
  T *sm = reinterpret_cast<T *>(smem);
  T *r0 = sm + G::R0;
  T *r1 = sm + G::R1;
  T *r2 = sm + G::R2;
  int *xs = reinterpret_cast<int *>(sm + G::END);  // wrapped x of theta^n-region columns
  int *ys = xs + G::W(0);                          // wrapped y of its rows
  const int tid = threadIdx.x;
  int bid = blockIdx.x;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * G::BX, y0 = by * G::BY;
  const int z0 = bz * p.zchunk;
  const int L = min(p.zchunk, p.nz - z0);
  const int nz = p.nz;
  const unsigned nx = (unsigned)p.nx, pln = nx * (unsigned)p.ny;
  for (int i = tid; i < G::W(0); i += NT) xs[i] = wrapn(x0 - 6 + i, p.nx);
  for (int j = tid; j < G::H(0); j += NT) ys[j] = wrapn(y0 - 6 + j, p.ny);
  __syncthreads();
  // theta^n planes z0-6 .. z0-2 into ring slots 0 .. 4; plane z0-1 is
  // copied asynchronously into slot 5
  auto zoff = [&](int q) { return (unsigned)wrapn(q, nz) * pln; };
  auto fetch = [&](int q, int slot) {
    const unsigned zo = zoff(q);
    T *dst = r0 + slot * N0;
    for (int it = tid; it < N0; it += NT) {
      const int jr = it / G::W(0), ic = it - jr * G::W(0);
      cp_async(dst + it, p.x + ((unsigned)xs[ic] + (unsigned)ys[jr] * nx + zo));
    }
  };
  for (int r = 0; r < NRING; ++r) {
    const unsigned zo = zoff(z0 - 6 + r);
    for (int it = tid; it < N0; it += NT) {
      const int jr = it / G::W(0), ic = it - jr * G::W(0);
      r0[r * N0 + it] = p.x[(unsigned)xs[ic] + (unsigned)ys[jr] * nx + zo];
    }
  }
  fetch(z0 - 1, NRING);
  cp_commit();
  __syncthreads();

  Stage<T, LIM, 1> s1;
  Stage<T, LIM, 2> s2;
  Stage<T, LIM, 3> s3;
  const int iters = L + PRO;
  s1.load_u(p, xs, ys, zoff(z0 - 4));
  for (int t = 0; t < iters; ++t) {
    const bool v1 = t < L + 8, v2 = t >= 5 && t < L + 9, v3 = t >= 10;
    const bool vl = t <= L + 5;
    const int q1 = z0 - 4 + t, q2 = z0 - 7 + t, q3 = z0 - 10 + t;
    // ring planes: theta^n plane q1+d in slot (t+2+d) % 6, theta^1 plane
    // q2+d in slot (t-3+d) % 5, theta^2 plane q3+d in slot (t-8+d) % 5
    auto P0 = [&](int d) { return r0 + ((t + 2 + d) % NRING0) * N0; };
    auto P1 = [&](int d) { return r1 + ((t - 3 + d) % NRING) * N1; };
    auto P2 = [&](int d) { return r2 + ((t - 8 + d) % NRING) * N2; };
    // theta^n plane z0+t (read from iteration t+2 on) into the slot of plane
    // z0-6+t, which this iteration's faces do not read (except at t = 0,
    // where the copy starts after the face phase); one commit group per
    // iteration, waited for one iteration later
    if (t > 0) {
      if (vl) fetch(z0 + t, t % NRING0);
      cp_commit();
    }
    if (p.combine) {
      if (v2) s2.load_thn(p, xs, ys, zoff(q2));
      if (v3) s3.load_thn(p, xs, ys, zoff(q3));
    }
    // ------------------------------------------------------------ faces
    if (v1) {
      s1.xy_faces(p, P0(0), sm + G::FX1, sm + G::FY1);
      if (p.az) {
        if (t == 0) s1.first_z(p, P0(-2), P0(-1), P0(0), P0(1), xs, ys, zoff(q1 - 1));
        s1.z_faces(P0(-1), P0(0), P0(1), P0(2), s1.uzr, s1.znew);
      }
    }
    if (v2) {
      s2.xy_faces(p, P1(0), sm + G::FX2, sm + G::FY2);
      if (p.az) {
        if (t == 5) s2.first_z(p, P1(-2), P1(-1), P1(0), P1(1), xs, ys, zoff(q2 - 1));
        s2.z_faces(P1(-1), P1(0), P1(1), P1(2), s2.uzr, s2.znew);
      }
    }
    if (v3) {
      s3.xy_faces(p, P2(0), sm + G::FX3, sm + G::FY3);
      if (p.az) {
        if (t == 10) s3.first_z(p, P2(-2), P2(-1), P2(0), P2(1), xs, ys, zoff(q3 - 1));
        s3.z_faces(P2(-1), P2(0), P2(1), P2(2), s3.uzr, s3.znew);
      }
    }
    // velocities of the next iteration's planes
    if (t + 1 < L + 8) s1.load_u(p, xs, ys, zoff(q1 + 1));
    if (t + 1 >= 5 && t + 1 < L + 9) s2.load_u(p, xs, ys, zoff(q2 + 1));
    if (t + 1 >= 10 && t + 1 < iters) s3.load_u(p, xs, ys, zoff(q3 + 1));
    __syncthreads();
    if (t == 0) {
      fetch(z0, 0);
      cp_commit();
    }
    // ------------------------------------------------------------ cells
    if (v1) {
      s1.update(p, false, T(0), T(1), p.cx[0], p.cy[0], p.cz[0], P0(0), sm + G::FX1,
                sm + G::FY1, r1 + (t % NRING) * N1, nullptr, x0, y0);
      s1.rotate();
    }
    if (v2) {
      s2.update(p, p.combine != 0, p.a2, p.b2, p.cx[1], p.cy[1], p.cz[1], P1(0), sm + G::FX2,
                sm + G::FY2, r2 + ((t - 5) % NRING) * N2, nullptr, x0, y0);
      s2.rotate();
    }
    if (v3) {
      s3.update(p, p.combine != 0, p.a3, p.b3, p.cx[2], p.cy[2], p.cz[2], P2(0), sm + G::FX3,
                sm + G::FY3, nullptr, p.y + (unsigned)q3 * pln, x0, y0);
      s3.rotate();
    }
    cp_wait_prev();
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class T, int LIM>
cudaError_t launch_fused(const FParams<T> &p, unsigned grid, cudaStream_t st) {
  auto k = k_struct_rk3_fused<T, LIM>;
  const cudaError_t e = set_smem_limit(reinterpret_cast<const void *>(k), (int)Geo<T>::BYTES);
  if (e != cudaSuccess) return e;
  k<<<grid, Geo<T>::NT, Geo<T>::BYTES, st>>>(p);
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch_fused(int lim, const FParams<T> &p, unsigned grid, cudaStream_t st) {
  switch (lim) {
    case LIM_UPWIND: return launch_fused<T, LIM_UPWIND>(p, grid, st);
    case LIM_CENTRAL: return launch_fused<T, LIM_CENTRAL>(p, grid, st);
    case LIM_MINMOD: return launch_fused<T, LIM_MINMOD>(p, grid, st);
    case LIM_VANLEER: return launch_fused<T, LIM_VANLEER>(p, grid, st);
    case LIM_SUPERBEE: return launch_fused<T, LIM_SUPERBEE>(p, grid, st);
    case LIM_SMART: return launch_fused<T, LIM_SMART>(p, grid, st);
  }
  return cudaErrorInvalidValue;
}

// One launch: y = three stages applied to x (SSP-RK3 when rk == 3, three
// forward-Euler steps when rk == 1).
template <class T>
cudaError_t fused_launch_t(const fl_mesh *m, int lim, int rk, double dtime, const void *x,
                           void *y, const void *u, cudaStream_t st) {
  using G = Geo<T>;
  FParams<T> p;
  p.x = static_cast<const T *>(x);
  p.y = static_cast<T *>(y);
  const T *ub = static_cast<const T *>(u);
  p.ux = ub + m->u_off[0];
  p.uy = ub + m->u_off[1];
  p.uz = ub + m->u_off[2];
  p.nx = m->nx;
  p.ny = m->ny;
  p.nz = m->nz;
  p.ax = m->act[0];
  p.ay = m->act[1];
  p.az = m->act[2];
  p.combine = rk == 3;
  // SSP-RK3 (Shu-Osher): theta^1 = x + dt R(x); theta^2 = 3/4 x + 1/4 (theta^1
  // + dt R(theta^1)); y = 1/3 x + 2/3 (theta^2 + dt R(theta^2))
  const double bs[3] = {1.0, rk == 3 ? 0.25 : 1.0, rk == 3 ? 2.0 / 3.0 : 1.0};
  p.a2 = blend_a<T>(0.75, 0.25);
  p.b2 = (T)0.25;
  p.a3 = blend_a<T>(1.0 / 3.0, 2.0 / 3.0);
  p.b3 = (T)(2.0 / 3.0);
  for (int s = 0; s < 3; ++s) {
    const double sc = bs[s] * dtime;
    p.cx[s] = (T)(sc / m->hx);
    p.cy[s] = (T)(sc / m->hy);
    p.cz[s] = (T)(sc / m->hz);
  }
  p.tiles_x = (m->nx + G::BX - 1) / G::BX;
  p.tiles_y = (m->ny + G::BY - 1) / G::BY;
  const long long cols = (long long)p.tiles_x * p.tiles_y;
  if (set_smem_limit(reinterpret_cast<const void *>(&k_struct_rk3_fused<T, LIM_SUPERBEE>),
                     (int)G::BYTES) != cudaSuccess)
    return cudaErrorNotSupported;
  const int resident = resident_ctas(
      reinterpret_cast<const void *>(&k_struct_rk3_fused<T, LIM_SUPERBEE>), G::NT, G::BYTES);
  p.zchunk = pick_zchunk(cols, m->nz, resident, PRO);
  const long long grid = cols * ((m->nz + p.zchunk - 1) / p.zchunk);
  if (grid >= (1LL << 31)) return cudaErrorInvalidConfiguration;
  return dispatch_fused<T>(lim, p, (unsigned)grid, st);
}

}  // namespace

size_t struct_fused_smem_bytes(fl_dtype dt) {
  return dt == FL_F64 ? Geo<double>::BYTES : Geo<float>::BYTES;
}

cudaError_t struct_step_fused(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                              int64_t nsteps, void *theta, const void *u, void *Y,
                              cudaStream_t st) {
  const size_t bytes = (size_t)m->C * dsize(dt);
  // each launch covers one SSP-RK3 step or three Euler steps
  const int64_t per = rk == 3 ? 1 : 3;
  const int64_t launches = nsteps / per, rest = nsteps - launches * per;
  void *cur = theta, *oth = Y;
  for (int64_t n = 0; n < launches; ++n) {
    const cudaError_t e = dt == FL_F64
                              ? fused_launch_t<double>(m, lim, rk, dtime, cur, oth, u, st)
                              : fused_launch_t<float>(m, lim, rk, dtime, cur, oth, u, st);
    if (e != cudaSuccess) return e;
    void *tmp = cur;
    cur = oth;
    oth = tmp;
  }
  if (cur != theta) {
    const cudaError_t e = cudaMemcpyAsync(theta, cur, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  // the remaining Euler steps (fewer than three) run stage by stage
  if (rest > 0) return struct_step(m, lim, dt, 1, dtime, rest, theta, u, Y, nullptr, nullptr, st);
  return cudaSuccess;
}

}  // namespace fl
