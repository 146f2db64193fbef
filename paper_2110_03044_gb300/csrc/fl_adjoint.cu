// fl_adjoint.cu -- adjoint (transpose Jacobian) of the limited-convection
// stage on periodic Cartesian meshes, and the checkpointed reverse sweep of
// an Euler / SSP-RK3 rollout.
//
// The forward face value, linearised on the branch the forward evaluation
// takes (limited_face_lin, same bit-pattern tests as limited_face), is
//   theta_f ~ theta_C + s (alpha Delta_m + beta Delta_up)
// so a face m+1/2 with adjoint weight g = (A/V) u_f (mu_{m+1} - mu_m) -- the
// derivative of sum_c mu_c R_c with respect to its flux -- hands
//   s > 0 (C = m, up face m-1):  -beta g to m-1, (1-alpha+beta) g to m, alpha g to m+1
//   s < 0 (C = m+1, up face m+1): alpha g to m, (1-alpha+beta) g to m+1, -beta g to m+2
// Every cell therefore gathers from four faces per axis (m = i-2 .. i+1).
// The kernel mirrors the forward one: a 32 x 8 column per CTA streams through
// z; theta (3-cell halo) and mu (2-cell halo) of the current plane sit in
// shared memory; per-face data (g, alpha, beta, 1-alpha+beta, s) is computed
// once per face in shared memory (z faces in registers) and gathered.
//
// Stage adjoint (RK stage y = a thn + b (x + dt R(x))):
//   out = e1 v1 + e2 v2 + b mu + b dt R'(x)^T mu      (v1, v2 pointwise)
// fl_conv_limited_adjoint is the bare out = R'(x)^T mu.
//
// In the reverse sweep of a piecewise-linear limiter the recomputed forward
// stages store each face's branch code, and k_struct_adjoint_codes reads the
// codes instead of theta (no theta tile, no differences).  The reverse sweep
// of a face-based mesh runs the gather kernel of fl_unstructured.cu.
#include <cuda_runtime.h>

#include <cmath>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"
#include "fl_unstructured.h"

namespace fl {

fl_status check_buffer(const void *p, size_t bytes, const char *name);
fl_status check_mesh(const fl_mesh *m);
fl_status check_enums(int lim, fl_dtype dt);
fl_status check_cell_range(const fl_mesh *m, int64_t c_begin, int64_t c_end);
fl_status check_box(const fl_mesh *m, int y_begin, int y_end, int z_begin, int z_end);

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
#ifndef FL_ADJ_MINB
#define FL_ADJ_MINB 3
#endif

template <class T>
struct AParams {
  const T *x;    // forward stage input (theta)
  const T *mu;   // adjoint of the stage output
  const T *v1;   // optional pointwise terms
  const T *v2;
  T *out;        // may alias v1 / v2 (own cell only), never x or mu
  const T *u;
  int nx, ny, nz;
  int act_x, act_y, act_z;
  long long ux_off, uy_off, uz_off;
  long long plane;
  T cx, cy, cz;  // A/V per axis
  T e1, e2, b, bdt;
  const unsigned char *codes;  // branch codes of the forward stage (layout of u), or null
  int bare;      // 1: out = R'^T mu only
  int tiles_x, tiles_y, zchunk;
  int zlo, zhi;  // the tiles cover planes [zlo, zhi)
  int ylo, yhi;  // and rows [ylo, yhi) of them
};

// asynchronous global -> shared copy of one element (no register staging)
template <class T>
__device__ __forceinline__ void cp_async1(T *dst, const T *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Branch constants (alpha, beta, 1 - alpha + beta) of the piecewise-linear
// limiters for branch codes 1..4, as the top 16 bits of their IEEE patterns
// (every constant is a short binary fraction, so the remaining bits are
// zero), four to a 64-bit word.  Decoding is a shift and a mask on the
// integer pipe: a switch on the code compiled to per-lane indexed constant
// loads, which serialise whenever the lanes of a warp hold different codes.
// Code 0 (correction off) is alpha = beta = 0, 1 - alpha + beta = 1.
//   minmod   1: beta 1/2      2: alpha 1/2
//   superbee 1: beta 1   2: alpha 1/2   3: beta 1/2   4: alpha 1
//   SMART    1: alpha 2  2: beta 1      3: alpha 1/8, beta 3/8
//   central  1: alpha 1/2
template <class T, int LIM>
struct CoefTab {
  static constexpr unsigned long long AL = 0, BE = 0, C1 = 0;
};
template <int LIM>
struct CoefTab<float, LIM> {
  static constexpr unsigned long long AL =
      LIM == LIM_CENTRAL ? 0x3f00ull
      : LIM == LIM_MINMOD ? 0x3f000000ull
      : LIM == LIM_SUPERBEE ? 0x3f8000003f000000ull
      : LIM == LIM_SMART ? 0x00003e0000004000ull : 0ull;
  static constexpr unsigned long long BE =
      LIM == LIM_MINMOD ? 0x3f00ull
      : LIM == LIM_SUPERBEE ? 0x00003f0000003f80ull
      : LIM == LIM_SMART ? 0x00003ec03f800000ull : 0ull;
  static constexpr unsigned long long C1 =
      LIM == LIM_CENTRAL ? 0x3f00ull
      : LIM == LIM_MINMOD ? 0x3f003fc0ull
      : LIM == LIM_SUPERBEE ? 0x00003fc03f004000ull
      : LIM == LIM_SMART ? 0x00003fa04000bf80ull : 0ull;
  static constexpr unsigned ONE = 0x3f80u;
  __device__ __forceinline__ static unsigned bits(unsigned h) { return h << 16; }
};
template <int LIM>
struct CoefTab<double, LIM> {
  static constexpr unsigned long long AL =
      LIM == LIM_CENTRAL ? 0x3fe0ull
      : LIM == LIM_MINMOD ? 0x3fe00000ull
      : LIM == LIM_SUPERBEE ? 0x3ff000003fe00000ull
      : LIM == LIM_SMART ? 0x00003fc000004000ull : 0ull;
  static constexpr unsigned long long BE =
      LIM == LIM_MINMOD ? 0x3fe0ull
      : LIM == LIM_SUPERBEE ? 0x00003fe000003ff0ull
      : LIM == LIM_SMART ? 0x00003fd83ff00000ull : 0ull;
  static constexpr unsigned long long C1 =
      LIM == LIM_CENTRAL ? 0x3fe0ull
      : LIM == LIM_MINMOD ? 0x3fe03ff8ull
      : LIM == LIM_SUPERBEE ? 0x00003ff83fe04000ull
      : LIM == LIM_SMART ? 0x00003ff44000bff0ull : 0ull;
  static constexpr unsigned ONE = 0x3ff0u;
  __device__ __forceinline__ static unsigned long long bits(unsigned h) {
    return (unsigned long long)h << 48;
  }
};

// Per-face adjoint data: the weight g and the branch coefficients.  For the
// piecewise-linear limiters the coefficients are constants of the branch, so
// only a small branch code is kept (fewer registers for the z faces and less
// shared memory); van Leer keeps its computed alpha, beta, 1 - alpha + beta.
template <class T, int LIM>
struct FaceAdj {
  using Tab = CoefTab<T, LIM>;
  using U = typename FT<T>::U;
  T g;
  int code;  // bits 0-2: branch, bit 3: s > 0
  __device__ __forceinline__ bool sp() const { return (code & 8) != 0; }
  // IEEE bit patterns of the branch's alpha, beta, 1 - alpha + beta
  __device__ __forceinline__ U pick(unsigned long long tab, unsigned off) const {
    const int b = code & 7;
    const unsigned h = b ? (unsigned)(tab >> (16 * (b - 1))) & 0xFFFFu : off;
    return Tab::bits(h);
  }
  __device__ __forceinline__ U al() const { return pick(Tab::AL, 0u); }
  __device__ __forceinline__ U be() const { return pick(Tab::BE, 0u); }
  __device__ __forceinline__ U c1() const { return pick(Tab::C1, Tab::ONE); }
};

template <class T>
struct FaceAdj<T, LIM_VANLEER> {
  T g, a_, b_, c_;
  bool s_;
  __device__ __forceinline__ bool sp() const { return s_; }
  __device__ __forceinline__ T al() const { return a_; }
  __device__ __forceinline__ T be() const { return b_; }
  __device__ __forceinline__ T c1() const { return c_; }
};

// Shared-memory face table in structure-of-arrays form (consecutive faces of
// a row are read by consecutive threads: one 8-byte word per thread, no bank
// conflicts).
template <class T, int LIM, int N>
struct FaceSmem {
  T g[N];
  int code[N];
  __device__ __forceinline__ void put(int i, const FaceAdj<T, LIM> &f) {
    g[i] = f.g;
    code[i] = f.code;
  }
  __device__ __forceinline__ FaceAdj<T, LIM> get(int i) const {
    FaceAdj<T, LIM> f;
    f.g = g[i];
    f.code = code[i];
    return f;
  }
};

template <class T, int N>
struct FaceSmem<T, LIM_VANLEER, N> {
  T g[N], a[N], b[N], c[N];
  unsigned char s[N];
  __device__ __forceinline__ void put(int i, const FaceAdj<T, LIM_VANLEER> &f) {
    g[i] = f.g;
    a[i] = f.a_;
    b[i] = f.b_;
    c[i] = f.c_;
    s[i] = f.s_;
  }
  __device__ __forceinline__ FaceAdj<T, LIM_VANLEER> get(int i) const {
    FaceAdj<T, LIM_VANLEER> f;
    f.g = g[i];
    f.a_ = a[i];
    f.b_ = b[i];
    f.c_ = c[i];
    f.s_ = s[i] != 0;
    return f;
  }
};

// c is the axis coefficient A/V; with PRE the velocities arrive already
// multiplied by it (one product per face saved in every adjoint stage)
template <class T, int LIM, bool PRE>
__device__ __forceinline__ FaceAdj<T, LIM> face_adj(T u, T a, T dm1, T dp1, T mu0, T mu1, T c) {
  using F = FT<T>;
  FaceAdj<T, LIM> r;
  const bool sp = upwind_positive(u);
  const T b = sp ? dm1 : dp1;
  if constexpr (LIM == LIM_VANLEER) {
    limited_face_lin<T, LIM>(a, b, r.a_, r.b_, r.c_);
    r.s_ = sp;
  } else {
    r.code = lin_code<T, LIM>(a, b) | (sp ? 8 : 0);
  }
  r.g = PRE ? F::mul(u, F::sub(mu1, mu0)) : F::mul(F::mul(c, u), F::sub(mu1, mu0));
  return r;
}

// contribution of the four faces m = i-2 .. i+1 of an axis to cell i
template <class T, int LIM>
__device__ __forceinline__ T gather4(T acc, const FaceAdj<T, LIM> &fm2, const FaceAdj<T, LIM> &fm1,
                                     const FaceAdj<T, LIM> &f0, const FaceAdj<T, LIM> &fp1) {
  using F = FT<T>;
  if constexpr (LIM == LIM_VANLEER) {
    acc = F::fma(f0.sp() ? f0.c1() : f0.al(), f0.g, acc);     // face i   (cell i is m)
    acc = F::fma(fm1.sp() ? fm1.al() : fm1.c1(), fm1.g, acc);  // face i-1 (cell i is m+1)
    if (fp1.sp()) acc = F::fma(-fp1.be(), fp1.g, acc);         // face i+1, s > 0: cell i is m-1
    if (!fm2.sp()) acc = F::fma(-fm2.be(), fm2.g, acc);        // face i-2, s < 0: cell i is m+2
  } else {
    // branch-free, with every coefficient (its sign, and 0 for a face that
    // does not reach cell i) formed on the integer pipe: on plain values the
    // compiler selected and negated them with FP64 operations.  (A
    // warp-uniform vote to skip the fma of a face no lane needs was
    // if-converted into an fma and a select: no FP64 saved.)
    using U = typename F::U;
    U c[4];
    c[0] = f0.sp() ? f0.c1() : f0.al();
    c[1] = fm1.sp() ? fm1.al() : fm1.c1();
    c[2] = fp1.sp() ? fp1.be() ^ F::SIGN : U(0);
    c[3] = fm2.sp() ? U(0) : fm2.be() ^ F::SIGN;
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = F::opaque(c[k]);
    acc = F::fma(F::val(c[0]), f0.g, acc);
    acc = F::fma(F::val(c[1]), fm1.g, acc);
    acc = F::fma(F::val(c[2]), fp1.g, acc);
    acc = F::fma(F::val(c[3]), fm2.g, acc);
  }
  return acc;
}

template <class T, int LIM, bool PRE>
__global__ void __launch_bounds__(TX *TY, FL_ADJ_MINB) k_struct_adjoint(const AParams<T> p) {
  using F = FT<T>;
  constexpr int NT = TX * TY;
  constexpr int SWT = TX + 6;  // theta row pitch (halo 3)
  constexpr int SWM = TX + 4;  // mu row pitch (halo 2)
  constexpr int NXF = TX + 3;  // x faces per row: m = x0-2 .. x0+TX
  constexpr int NYF = TY + 3;  // y faces per column: m = y0-2 .. y0+TY
  __shared__ T s_th[(TY + 6) * SWT];
  __shared__ T s_mu[(TY + 4) * SWM];
  __shared__ T s_dx[TY * (TX + 5)];  // Delta of x faces x0-3 .. x0+TX+1
  __shared__ T s_dy[(TY + 5) * TX];  // Delta of y faces y0-3 .. y0+TY+1
  __shared__ FaceSmem<T, LIM, TY * NXF> s_fx;
  __shared__ FaceSmem<T, LIM, NYF * TX> s_fy;
  // u of the x faces (m = x0-2 .. x0+TX) and y faces (m = y0-2 .. y0+TY) of
  // a plane, double-buffered: plane k+1 is copied in while k is processed
  __shared__ T s_uxb[2][TY * NXF];
  __shared__ T s_uyb[2][NYF * TX];
  __shared__ int s_wx[TX + 6];
  __shared__ int s_wy[TY + 6];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  int bid = blockIdx.x;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = p.ylo + by * TY;
  const int z0 = p.zlo + bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.zhi);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (tid < TX + 6) s_wx[tid] = wrapi(x0 - 3 + tid, nx);
  if (tid < TY + 6) s_wy[tid] = wrapi(y0 - 3 + tid, ny);
  __syncthreads();
  const bool valid = (x0 + tx < nx) && (y0 + ty < p.yhi);
  // wrap table index w <-> coordinate x0-3+w
  const long long col = (long long)s_wx[tx + 3] + (long long)nx * s_wy[ty + 3];

  // halo cells: theta 3 wide (6 per row, 6 rows), mu 2 wide
  int th_slot = -1, mu_slot = -1;
  long long th_off = 0, mu_off = 0;
  {
    constexpr int NHX = 6 * TY, NHT = NHX + 6 * TX;
    static_assert(NHT <= NT, "theta halo exceeds threads");
    if (tid < NHX) {
      const int r = tid / 6, k6 = tid % 6;
      const int c = (k6 < 3) ? k6 : (TX + k6);  // 0,1,2, TX+3,TX+4,TX+5
      th_slot = (r + 3) * SWT + c;
      th_off = (long long)s_wx[c] + (long long)nx * s_wy[r + 3];
    } else if (tid < NHT) {
      const int t = tid - NHX;
      const int k6 = t / TX, c = t % TX;
      const int r = (k6 < 3) ? k6 : (TY + k6);
      th_slot = r * SWT + c + 3;
      th_off = (long long)s_wx[c + 3] + (long long)nx * s_wy[r];
    }
    constexpr int NMX = 4 * TY, NMT = NMX + 4 * TX;
    static_assert(NMT <= NT, "mu halo exceeds threads");
    if (tid < NMX) {
      const int r = tid >> 2, k4 = tid & 3;
      const int c = (k4 < 2) ? k4 : (TX + k4);  // mu columns 0,1,TX+2,TX+3
      mu_slot = (r + 2) * SWM + c;
      mu_off = (long long)s_wx[c + 1] + (long long)nx * s_wy[r + 3];
    } else if (tid < NMT) {
      const int t = tid - NMX;
      const int k4 = t / TX, c = t % TX;
      const int r = (k4 < 2) ? k4 : (TY + k4);
      mu_slot = r * SWM + c + 2;
      mu_off = (long long)s_wx[c + 3] + (long long)nx * s_wy[r + 1];
    }
  }
  const bool need_x = p.act_x, need_y = p.act_y, need_z = p.act_z;
  // u of the plane's faces, copied one plane ahead (cp.async): every thread
  // its own +x and +y face; threads tid < 3 (TX + TY) one halo face each (x
  // faces x0-2, x0-1, x0+TX of every row, y faces y0-2, y0-1, y0+TY of every
  // column)
  int hu_slot = -1;
  long long hu_off = 0;
  bool hu_x = false;
  {
    constexpr int NUX = 3 * TY, NUT = NUX + 3 * TX;
    static_assert(NUT <= NT, "u halo exceeds threads");
    if (tid < NUX) {
      if (need_x) {
        const int r = tid / 3, k3 = tid % 3;
        const int q = (k3 < 2) ? k3 : TX + 2;  // face x0-2+q
        hu_slot = r * NXF + q;
        hu_off = p.ux_off + s_wx[q + 1] + (long long)nx * s_wy[r + 3];
        hu_x = true;
      }
    } else if (tid < NUT) {
      if (need_y) {
        const int t = tid - NUX;
        const int k3 = t / TX, c = t % TX;
        const int r = (k3 < 2) ? k3 : TY + 2;  // face y0-2+r
        hu_slot = r * TX + c;
        hu_off = p.uy_off + s_wx[c + 3] + (long long)nx * s_wy[r + 1];
      }
    }
  }
  auto load_u = [&](long long pk, int buf) {
    if (need_x) cp_async1(&s_uxb[buf][ty * NXF + tx + 2], p.u + p.ux_off + col + pk);
    if (need_y) cp_async1(&s_uyb[buf][(ty + 2) * TX + tx], p.u + p.uy_off + col + pk);
    if (hu_slot >= 0) cp_async1(hu_x ? &s_uxb[buf][hu_slot] : &s_uyb[buf][hu_slot], p.u + hu_off + pk);
    cp_async_commit();
  };
  load_u(p.plane * z0, z0 & 1);

  // ---- z prologue: faces z0-2, z0-1, z0 and the column window
  T th_k, th_k1, th_k2, d_k = T(0), d_k1 = T(0), mu_k, mu_k1 = T(0);
  FaceAdj<T, LIM> zf_m2{}, zf_m1{}, zf_0{};
  auto X = [&](int k) { return p.x[col + p.plane * wrapi(k, nz)]; };
  auto MU = [&](int k) { return p.mu[col + p.plane * wrapi(k, nz)]; };
  if (need_z) {
    const T tm3 = X(z0 - 3), tm2 = X(z0 - 2), tm1 = X(z0 - 1);
    th_k = X(z0);
    th_k1 = X(z0 + 1);
    th_k2 = X(z0 + 2);
    const T dm3 = F::sub(tm2, tm3), dm2 = F::sub(tm1, tm2), dm1 = F::sub(th_k, tm1);
    d_k = F::sub(th_k1, th_k);
    d_k1 = F::sub(th_k2, th_k1);
    const T mm2 = MU(z0 - 2), mm1 = MU(z0 - 1);
    mu_k = MU(z0);
    mu_k1 = MU(z0 + 1);
    const T *uz = p.u + p.uz_off + col;
    zf_m2 = face_adj<T, LIM, PRE>(uz[p.plane * wrapi(z0 - 2, nz)], dm2, dm3, dm1, mm2, mm1, p.cz);
    zf_m1 = face_adj<T, LIM, PRE>(uz[p.plane * wrapi(z0 - 1, nz)], dm1, dm2, d_k, mm1, mu_k, p.cz);
    zf_0 = face_adj<T, LIM, PRE>(uz[p.plane * z0], d_k, dm1, d_k1, mu_k, mu_k1, p.cz);
  } else {
    th_k = th_k1 = th_k2 = p.x[col];
    mu_k = p.mu[col];
  }

  for (int k = z0; k < z1; ++k) {
    const long long pk = p.plane * k;
    T th_k3 = T(0), mu_k2 = T(0), uz1 = T(0);
    if (need_z) {
      th_k3 = X(k + 3);
      mu_k2 = MU(k + 2);
      uz1 = p.u[p.uz_off + col + p.plane * wrapi(k + 1, nz)];
    }
    const T hv_t = (th_slot >= 0) ? p.x[th_off + pk] : T(0);
    const T hv_m = (mu_slot >= 0) ? p.mu[mu_off + pk] : T(0);
    T v1 = T(0), v2 = T(0);
    if (!p.bare && valid) {
      if (p.v1) v1 = p.v1[col + pk];
      if (p.v2) v2 = p.v2[col + pk];
    }
    s_th[(ty + 3) * SWT + tx + 3] = th_k;
    s_mu[(ty + 2) * SWM + tx + 2] = mu_k;
    if (th_slot >= 0) s_th[th_slot] = hv_t;
    if (mu_slot >= 0) s_mu[mu_slot] = hv_m;
    // this plane's u copies are complete (the barrier publishes them); the
    // next plane's go to the other buffer, last read before the previous
    // plane's final barrier
    cp_async_wait_all();
    if (k + 1 < z1) load_u(pk + p.plane, (k + 1) & 1);
    const T *s_ux = s_uxb[k & 1];
    const T *s_uy = s_uyb[k & 1];
    __syncthreads();
    // ---------------------------------------------- differences
    if (need_x) {
      for (int it = tid; it < TY * (TX + 5); it += NT) {
        const int r = it / (TX + 5), q = it - r * (TX + 5);  // face x0-3+q
        const T *row = &s_th[(r + 3) * SWT];
        s_dx[it] = F::sub(row[q + 1], row[q]);
      }
    }
    if (need_y) {
      for (int it = tid; it < (TY + 5) * TX; it += NT) {
        const int r = it / TX, c = it - r * TX;  // face y0-3+r
        s_dy[it] = F::sub(s_th[(r + 1) * SWT + c + 3], s_th[r * SWT + c + 3]);
      }
    }
    T d_k2 = T(0);
    if (need_z) d_k2 = F::sub(th_k3, th_k2);
    __syncthreads();
    // ---------------------------------------------- face data
    if (need_x) {
      for (int it = tid; it < TY * NXF; it += NT) {
        const int r = it / NXF, q = it - r * NXF;  // face m = x0-2+q
        const T uf = s_ux[it];
        const T *dr = &s_dx[r * (TX + 5)];  // Delta_m at q+1
        const T *mr = &s_mu[(r + 2) * SWM];  // mu_m at column q
        s_fx.put(it, face_adj<T, LIM, PRE>(uf, dr[q + 1], dr[q], dr[q + 2], mr[q], mr[q + 1], p.cx));
      }
    }
    if (need_y) {
      for (int it = tid; it < NYF * TX; it += NT) {
        const int r = it / TX, c = it - r * TX;  // face m = y0-2+r
        const T uf = s_uy[it];
        s_fy.put(it, face_adj<T, LIM, PRE>(uf, s_dy[(r + 1) * TX + c], s_dy[r * TX + c],
                                           s_dy[(r + 2) * TX + c], s_mu[r * SWM + c + 2],
                                           s_mu[(r + 1) * SWM + c + 2], p.cy));
      }
    }
    FaceAdj<T, LIM> zf_1{};
    if (need_z) zf_1 = face_adj<T, LIM, PRE>(uz1, d_k1, d_k, d_k2, mu_k1, mu_k2, p.cz);
    __syncthreads();
    // ---------------------------------------------- gather + combine
    if (valid) {
      T acc = T(0);
      if (need_x) {
        const int i = ty * NXF + tx;  // faces i-2 .. i+1
        acc = gather4(acc, s_fx.get(i), s_fx.get(i + 1), s_fx.get(i + 2), s_fx.get(i + 3));
      }
      if (need_y) {
        acc = gather4(acc, s_fy.get(ty * TX + tx), s_fy.get((ty + 1) * TX + tx),
                      s_fy.get((ty + 2) * TX + tx), s_fy.get((ty + 3) * TX + tx));
      }
      if (need_z) acc = gather4(acc, zf_m2, zf_m1, zf_0, zf_1);
      T o;
      if (p.bare) {
        o = acc;
      } else {
        o = F::fma(p.bdt, acc, F::mul(p.b, mu_k));
        if (p.v1) o = F::fma(p.e1, v1, o);
        if (p.v2) o = F::fma(p.e2, v2, o);
      }
      p.out[col + pk] = o;
    }
    // ---------------------------------------------- rotate
    if (need_z) {
      zf_m2 = zf_m1;
      zf_m1 = zf_0;
      zf_0 = zf_1;
      th_k = th_k1;
      th_k1 = th_k2;
      th_k2 = th_k3;
      d_k = d_k1;
      d_k1 = d_k2;
      mu_k = mu_k1;
      mu_k1 = mu_k2;
    } else if (k + 1 < z1) {
      th_k = p.x[col + p.plane * (k + 1)];
      mu_k = p.mu[col + p.plane * (k + 1)];
    }
  }
}


// The stage adjoint from stored branch codes: the forward stage that read x
// (run with codes on, in the reverse sweep's recomputation) left the branch
// code of every face, so this kernel needs neither x nor its differences --
// per face only g = w (mu_{m+1} - mu_m) and the code.  Same tiles, halos,
// gather and combination as k_struct_adjoint; two barriers per plane.
// Piecewise-linear limiters only (u holds w, the pre-scaled velocity).
template <class T, int LIM>
__global__ void __launch_bounds__(TX *TY, 4) k_struct_adjoint_codes(const AParams<T> p) {
  using F = FT<T>;
  constexpr int NT = TX * TY;
  constexpr int SWM = TX + 4;  // mu row pitch (halo 2)
  constexpr int NXF = TX + 3;  // x faces per row: m = x0-2 .. x0+TX
  constexpr int NYF = TY + 3;  // y faces per column: m = y0-2 .. y0+TY
  __shared__ T s_mu[(TY + 4) * SWM];
  __shared__ FaceSmem<T, LIM, TY * NXF> s_fx;
  __shared__ FaceSmem<T, LIM, NYF * TX> s_fy;
  __shared__ T s_uxb[2][TY * NXF];
  __shared__ T s_uyb[2][NYF * TX];
  __shared__ unsigned char s_cx[TY * NXF];
  __shared__ unsigned char s_cy[NYF * TX];
  __shared__ int s_wx[TX + 6];
  __shared__ int s_wy[TY + 6];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  int bid = blockIdx.x;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = p.ylo + by * TY;
  const int z0 = p.zlo + bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.zhi);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (tid < TX + 6) s_wx[tid] = wrapi(x0 - 3 + tid, nx);
  if (tid < TY + 6) s_wy[tid] = wrapi(y0 - 3 + tid, ny);
  __syncthreads();
  const bool valid = (x0 + tx < nx) && (y0 + ty < p.yhi);
  // addressing: 64-bit base pointers per stream, 32-bit offsets (cell and
  // plane offsets are below n_cells < 2^31): one wide multiply-add a load
  const unsigned plane = (unsigned)p.plane;
  const unsigned col = (unsigned)s_wx[tx + 3] + (unsigned)nx * (unsigned)s_wy[ty + 3];
  const T *__restrict__ Ux = p.u + p.ux_off;
  const T *__restrict__ Uy = p.u + p.uy_off;
  const T *__restrict__ Uz = p.u + p.uz_off;
  const unsigned char *__restrict__ Cx = p.codes + p.ux_off;
  const unsigned char *__restrict__ Cy = p.codes + p.uy_off;
  const unsigned char *__restrict__ Cz = p.codes + p.uz_off;
  const bool need_x = p.act_x, need_y = p.act_y, need_z = p.act_z;

  // mu halo (2 wide)
  int mu_slot = -1;
  unsigned mu_off = 0;
  {
    constexpr int NMX = 4 * TY, NMT = NMX + 4 * TX;
    static_assert(NMT <= NT, "mu halo exceeds threads");
    if (tid < NMX) {
      const int r = tid >> 2, k4 = tid & 3;
      const int c = (k4 < 2) ? k4 : (TX + k4);
      mu_slot = (r + 2) * SWM + c;
      mu_off = (unsigned)s_wx[c + 1] + (unsigned)nx * (unsigned)s_wy[r + 3];
    } else if (tid < NMT) {
      const int t = tid - NMX;
      const int k4 = t / TX, c = t % TX;
      const int r = (k4 < 2) ? k4 : (TY + k4);
      mu_slot = r * SWM + c + 2;
      mu_off = (unsigned)s_wx[c + 3] + (unsigned)nx * (unsigned)s_wy[r + 1];
    }
  }
  // faces of the plane: every thread its own +x and +y face, threads
  // tid < 3 (TX + TY) one halo face each (u by cp.async, codes by registers)
  int hu_slot = -1;
  unsigned hu_off = 0;
  bool hu_x = false;
  {
    constexpr int NUX = 3 * TY, NUT = NUX + 3 * TX;
    static_assert(NUT <= NT, "u halo exceeds threads");
    if (tid < NUX) {
      if (need_x) {
        const int r = tid / 3, k3 = tid % 3;
        const int q = (k3 < 2) ? k3 : TX + 2;
        hu_slot = r * NXF + q;
        hu_off = (unsigned)s_wx[q + 1] + (unsigned)nx * (unsigned)s_wy[r + 3];
        hu_x = true;
      }
    } else if (tid < NUT) {
      if (need_y) {
        const int t = tid - NUX;
        const int k3 = t / TX, c = t % TX;
        const int r = (k3 < 2) ? k3 : TY + 2;
        hu_slot = r * TX + c;
        hu_off = (unsigned)s_wx[c + 3] + (unsigned)nx * (unsigned)s_wy[r + 1];
      }
    }
  }
  unsigned cx_n = 0, cy_n = 0, ch_n = 0;
  auto load_face = [&](unsigned pk, int buf) {
    if (need_x) {
      cp_async1(&s_uxb[buf][ty * NXF + tx + 2], Ux + (col + pk));
      cx_n = Cx[col + pk];
    }
    if (need_y) {
      cp_async1(&s_uyb[buf][(ty + 2) * TX + tx], Uy + (col + pk));
      cy_n = Cy[col + pk];
    }
    if (hu_slot >= 0) {
      cp_async1(hu_x ? &s_uxb[buf][hu_slot] : &s_uyb[buf][hu_slot],
                (hu_x ? Ux : Uy) + (hu_off + pk));
      ch_n = (hu_x ? Cx : Cy)[hu_off + pk];
    }
    cp_async_commit();
  };
  load_face(plane * (unsigned)z0, z0 & 1);

  // ---- z prologue: faces z0-2, z0-1, z0 from the mu column and the codes
  T mu_k, mu_k1 = T(0);
  FaceAdj<T, LIM> zf_m2{}, zf_m1{}, zf_0{};
  auto MU = [&](int k) { return p.mu[col + plane * (unsigned)wrapi(k, nz)]; };
  auto ZF = [&](int k, T m0, T m1) {
    const unsigned i = col + plane * (unsigned)wrapi(k, nz);
    FaceAdj<T, LIM> f;
    f.g = F::mul(Uz[i], F::sub(m1, m0));
    f.code = Cz[i];
    return f;
  };
  if (need_z) {
    const T mm2 = MU(z0 - 2), mm1 = MU(z0 - 1);
    mu_k = MU(z0);
    mu_k1 = MU(z0 + 1);
    zf_m2 = ZF(z0 - 2, mm2, mm1);
    zf_m1 = ZF(z0 - 1, mm1, mu_k);
    zf_0 = ZF(z0, mu_k, mu_k1);
  } else {
    mu_k = p.mu[col];
  }

  for (int k = z0; k < z1; ++k) {
    const unsigned pk = plane * (unsigned)k;
    T mu_k2 = T(0);
    if (need_z) mu_k2 = MU(k + 2);
    const T hv_m = (mu_slot >= 0) ? p.mu[mu_off + pk] : T(0);
    T v1 = T(0), v2 = T(0);
    if (!p.bare && valid) {
      if (p.v1) v1 = p.v1[col + pk];
      if (p.v2) v2 = p.v2[col + pk];
    }
    s_mu[(ty + 2) * SWM + tx + 2] = mu_k;
    if (mu_slot >= 0) s_mu[mu_slot] = hv_m;
    if (need_x) s_cx[ty * NXF + tx + 2] = (unsigned char)cx_n;
    if (need_y) s_cy[(ty + 2) * TX + tx] = (unsigned char)cy_n;
    if (hu_slot >= 0) {
      if (hu_x) s_cx[hu_slot] = (unsigned char)ch_n;
      else s_cy[hu_slot] = (unsigned char)ch_n;
    }
    cp_async_wait_all();
    if (k + 1 < z1) load_face(pk + plane, (k + 1) & 1);
    const T *s_ux = s_uxb[k & 1];
    const T *s_uy = s_uyb[k & 1];
    FaceAdj<T, LIM> zf_1{};
    if (need_z) zf_1 = ZF(k + 1, mu_k1, mu_k2);
    __syncthreads();
    // ---------------------------------------------- face data
    if (need_x) {
      for (int it = tid; it < TY * NXF; it += NT) {
        const int r = it / NXF, q = it - r * NXF;  // face m = x0-2+q
        const T *mr = &s_mu[(r + 2) * SWM];
        FaceAdj<T, LIM> f;
        f.g = F::mul(s_ux[it], F::sub(mr[q + 1], mr[q]));
        f.code = s_cx[it];
        s_fx.put(it, f);
      }
    }
    if (need_y) {
      for (int it = tid; it < NYF * TX; it += NT) {
        const int r = it / TX, c = it - r * TX;  // face m = y0-2+r
        FaceAdj<T, LIM> f;
        f.g = F::mul(s_uy[it], F::sub(s_mu[(r + 1) * SWM + c + 2], s_mu[r * SWM + c + 2]));
        f.code = s_cy[it];
        s_fy.put(it, f);
      }
    }
    __syncthreads();
    // ---------------------------------------------- gather + combine
    if (valid) {
      T acc = T(0);
      if (need_x) {
        const int i = ty * NXF + tx;
        acc = gather4(acc, s_fx.get(i), s_fx.get(i + 1), s_fx.get(i + 2), s_fx.get(i + 3));
      }
      if (need_y) {
        acc = gather4(acc, s_fy.get(ty * TX + tx), s_fy.get((ty + 1) * TX + tx),
                      s_fy.get((ty + 2) * TX + tx), s_fy.get((ty + 3) * TX + tx));
      }
      if (need_z) acc = gather4(acc, zf_m2, zf_m1, zf_0, zf_1);
      T o;
      if (p.bare) {
        o = acc;
      } else {
        o = F::fma(p.bdt, acc, F::mul(p.b, mu_k));
        if (p.v1) o = F::fma(p.e1, v1, o);
        if (p.v2) o = F::fma(p.e2, v2, o);
      }
      p.out[col + pk] = o;
    }
    if (need_z) {
      zf_m2 = zf_m1;
      zf_m1 = zf_0;
      zf_0 = zf_1;
      mu_k = mu_k1;
      mu_k1 = mu_k2;
    } else if (k + 1 < z1) {
      mu_k = p.mu[col + plane * (unsigned)(k + 1)];
    }
  }
}

template <class T>
cudaError_t run_adj_t(const fl_mesh *m, int lim, const AdjArgs &s, cudaStream_t st) {
  AParams<T> p;
  p.x = static_cast<const T *>(s.x);
  p.mu = static_cast<const T *>(s.mu);
  p.v1 = static_cast<const T *>(s.v1);
  p.v2 = static_cast<const T *>(s.v2);
  p.out = static_cast<T *>(s.out);
  p.u = static_cast<const T *>(s.cu ? s.cu : s.u);
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
  p.cx = (T)(1.0 / m->hx);
  p.cy = (T)(1.0 / m->hy);
  p.cz = (T)(1.0 / m->hz);
  p.e1 = (T)s.e1;
  p.e2 = (T)s.e2;
  p.b = (T)s.b;
  p.bdt = (T)(s.cu_dt ? s.b : s.b * s.dt);
  p.bare = s.bare;
  p.codes = static_cast<const unsigned char *>(s.codes);
  p.tiles_x = (m->nx + TX - 1) / TX;
  p.ylo = s.yhi < 0 ? 0 : s.ylo;
  p.yhi = s.yhi < 0 ? m->ny : s.yhi;
  p.tiles_y = (p.yhi - p.ylo + TY - 1) / TY;
  p.zlo = s.zhi < 0 ? 0 : s.zlo;
  p.zhi = s.zhi < 0 ? m->nz : s.zhi;
  const int nzr = p.zhi - p.zlo;
  const long long cols = (long long)p.tiles_x * p.tiles_y;
  if (s.codes != nullptr && s.cu != nullptr && lim != LIM_VANLEER) {
    // the stage's branch codes are stored: no theta, no differences
    const int res = resident_ctas(
        reinterpret_cast<const void *>(&k_struct_adjoint_codes<T, LIM_SUPERBEE>), TX * TY, 0);
    p.zchunk = pick_zchunk(cols, nzr, res, 2);
    const unsigned g = (unsigned)(cols * ((nzr + p.zchunk - 1) / p.zchunk));
    const dim3 blk(TX, TY);
    switch (lim) {
      case LIM_UPWIND: k_struct_adjoint_codes<T, LIM_UPWIND><<<g, blk, 0, st>>>(p); break;
      case LIM_CENTRAL: k_struct_adjoint_codes<T, LIM_CENTRAL><<<g, blk, 0, st>>>(p); break;
      case LIM_MINMOD: k_struct_adjoint_codes<T, LIM_MINMOD><<<g, blk, 0, st>>>(p); break;
      case LIM_SUPERBEE: k_struct_adjoint_codes<T, LIM_SUPERBEE><<<g, blk, 0, st>>>(p); break;
      case LIM_SMART: k_struct_adjoint_codes<T, LIM_SMART><<<g, blk, 0, st>>>(p); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const int resident = resident_ctas(
      reinterpret_cast<const void *>(&k_struct_adjoint<T, LIM_SUPERBEE, true>), TX * TY, 0);
  const int zchunk = pick_zchunk(cols, nzr, resident, 3);
  p.zchunk = zchunk;
  const int tz = (nzr + zchunk - 1) / zchunk;
  const unsigned grid = (unsigned)(cols * tz);
  const dim3 block(TX, TY);
#define FL_ADJ_CASE(L)                                                     \
  case L:                                                                  \
    if (s.cu) k_struct_adjoint<T, L, true><<<grid, block, 0, st>>>(p);     \
    else k_struct_adjoint<T, L, false><<<grid, block, 0, st>>>(p);         \
    break;
  switch (lim) {
    FL_ADJ_CASE(LIM_UPWIND)
    FL_ADJ_CASE(LIM_CENTRAL)
    FL_ADJ_CASE(LIM_MINMOD)
    FL_ADJ_CASE(LIM_VANLEER)
    FL_ADJ_CASE(LIM_SUPERBEE)
    FL_ADJ_CASE(LIM_SMART)
    default: return cudaErrorInvalidValue;
  }
#undef FL_ADJ_CASE
  return cudaGetLastError();
}

}  // namespace

cudaError_t struct_adjoint(const fl_mesh *m, int lim, fl_dtype dt, const AdjArgs &s,
                           cudaStream_t st) {
  return dt == FL_F64 ? run_adj_t<double>(m, lim, s, st) : run_adj_t<float>(m, lim, s, st);
}

// one stage adjoint on either kind of mesh
cudaError_t adjoint_any(const fl_mesh *m, int lim, fl_dtype dt, const AdjArgs &s, cudaStream_t st) {
  return m->kind == 1 ? unstruct_adjoint(m, lim, dt, s, st) : struct_adjoint(m, lim, dt, s, st);
}

// ------------------------------------------------------------- host side
size_t adjoint_ws_bytes(const fl_mesh *m, fl_dtype dt, int rk, int64_t nsteps, int64_t every) {
  const size_t one = align256((size_t)m->C * dsize(dt));
  const int S = (rk == 3) ? 3 : 1;
  const int64_t nck = (nsteps + every - 1) / every;
  const int64_t seg = (int64_t)S * every + 1;
  // checkpoints | segment stage states | 3 adjoint vectors | pre-scaled u_f |
  // branch codes of the segment's stages (one byte per face and stage)
  return one * (size_t)(nck + seg + 3) + align256((size_t)m->F * dsize(dt)) +
         align256((size_t)m->F * (size_t)(S * every));
}

}  // namespace fl

using namespace fl;

#define FL_TRY(expr)            \
  do {                          \
    fl_status s_ = (expr);      \
    if (s_ != FL_OK) return s_; \
  } while (0)

// One adjoint stage over planes [zlo, zhi) of a structured mesh or cells
// [clo, chi) of a local face-based mesh (a negative end: every plane / owned
// cell): the shared body of fl_step_rk_stage_adjoint and its _planes and
// _cells forms.
static fl_status stage_adjoint_planes(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                      int stage, double dtime, int ylo, int yhi, int zlo, int zhi,
                                      int64_t clo, int64_t chi, const void *x, const void *mu,
                                      const void *lam_a, const void *lam_b, void *out,
                                      const void *u_f, const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (stage < 0 || stage >= (rk == 3 ? 3 : 1))
    return fail(FL_EINVAL, "stage %d does not exist for rk_order %d", stage, rk);
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  const size_t es = dsize(dt), cb = (size_t)m->C * es;
  FL_TRY(check_buffer(x, cb, "x"));
  FL_TRY(check_buffer(mu, cb, "mu"));
  FL_TRY(check_buffer(out, cb, "out"));
  FL_TRY(check_buffer(u_f, (size_t)m->F * es, "u_f"));
  const bool blend = rk == 3 && stage == 0;
  if (blend) {
    FL_TRY(check_buffer(lam_a, cb, "lam_a"));
    FL_TRY(check_buffer(lam_b, cb, "lam_b"));
  }
  if (w_f != nullptr) {
    if (!(dtime > 0)) return fail(FL_EINVAL, "a pre-scaled velocity needs dt > 0");
    FL_TRY(check_buffer(w_f, (size_t)m->F * es, "w_f"));
  }
  if (m->C > 0) {
    const char *ob = static_cast<const char *>(out);
    for (const void *in : {x, mu}) {
      const char *ib = static_cast<const char *>(in);
      if (ob < ib + cb && ib < ob + cb)
        return fail(FL_EINVAL, "out overlaps x or mu (the stage reads their neighbours)");
    }
  }
  if (m->C == 0 || (zhi >= 0 && zhi == zlo) || (yhi >= 0 && yhi == ylo) ||
      (chi >= 0 && chi == clo))
    return FL_OK;
  if (m->kind == 1) FL_TRY(unstruct_adjoint_prepare(m));
  AdjArgs a;
  a.zlo = zlo;
  a.zhi = zhi;
  a.ylo = ylo;
  a.yhi = yhi;
  a.clo = clo;
  a.chi = chi;
  a.x = x;
  a.mu = mu;
  a.out = out;
  a.u = u_f;
  a.cu = w_f;
  a.cu_dt = w_f != nullptr;
  a.dt = dtime;
  a.b = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  if (blend) {
    // theta^n's weights in the later stages' blends: 1/3 in stage 2 (as the
    // forward kernels use it: 1 - RN(2/3) in the working precision) and 3/4
    // in stage 1
    a.v1 = lam_b;
    a.e1 = dt == FL_F64 ? blend_a<double>(1.0 / 3.0, 2.0 / 3.0)
                        : (double)blend_a<float>(1.0 / 3.0, 2.0 / 3.0);
    a.v2 = lam_a;
    a.e2 = 0.75;
  }
  const cudaError_t e = adjoint_any(m, lim, dt, a, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stage adjoint kernel");
  return FL_OK;
}

extern "C" {

fl_status fl_conv_limited_adjoint(const fl_mesh *m, fl_limiter lim, fl_dtype dt,
                                  const void *theta_c, const void *u_f, const void *lambda_rhs,
                                  void *lambda_theta, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(theta_c, m->C * es, "theta_c"));
  FL_TRY(check_buffer(u_f, m->F * es, "u_f"));
  FL_TRY(check_buffer(lambda_rhs, m->C * es, "lambda_rhs"));
  FL_TRY(check_buffer(lambda_theta, m->C * es, "lambda_theta"));
  if (lambda_theta == lambda_rhs || lambda_theta == theta_c)
    return fail(FL_EINVAL, "lambda_theta must not alias the inputs");
  if (m->C == 0) return FL_OK;
  if (m->kind == 1) FL_TRY(unstruct_adjoint_prepare(m));
  AdjArgs a;
  a.x = theta_c;
  a.mu = lambda_rhs;
  a.out = lambda_theta;
  a.u = u_f;
  a.bare = 1;
  cudaError_t e = adjoint_any(m, lim, dt, a, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel");
  return FL_OK;
}

fl_status fl_step_rk_stage_adjoint(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                   int stage, double dtime, const void *x, const void *mu,
                                   const void *lam_a, const void *lam_b, void *out,
                                   const void *u_f, const void *w_f, void *stream) {
  return stage_adjoint_planes(m, lim, dt, rk, stage, dtime, 0, -1, 0, -1, 0, -1, x, mu, lam_a,
                              lam_b, out, u_f, w_f, stream);
}

fl_status fl_step_rk_stage_adjoint_planes(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                          int stage, double dtime, int z_begin, int z_end,
                                          const void *x, const void *mu, const void *lam_a,
                                          const void *lam_b, void *out, const void *u_f,
                                          const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_box(m, 0, m->ny, z_begin, z_end));
  return stage_adjoint_planes(m, lim, dt, rk, stage, dtime, 0, -1, z_begin, z_end, 0, -1, x, mu,
                              lam_a, lam_b, out, u_f, w_f, stream);
}

fl_status fl_step_rk_stage_adjoint_box(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                       int stage, double dtime, int y_begin, int y_end,
                                       int z_begin, int z_end, const void *x, const void *mu,
                                       const void *lam_a, const void *lam_b, void *out,
                                       const void *u_f, const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_box(m, y_begin, y_end, z_begin, z_end));
  return stage_adjoint_planes(m, lim, dt, rk, stage, dtime, y_begin, y_end, z_begin, z_end, 0, -1,
                              x, mu, lam_a, lam_b, out, u_f, w_f, stream);
}

fl_status fl_step_rk_stage_adjoint_cells(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                         int stage, double dtime, int64_t c_begin, int64_t c_end,
                                         const void *x, const void *mu, const void *lam_a,
                                         const void *lam_b, void *out, const void *u_f,
                                         const void *w_f, void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_cell_range(m, c_begin, c_end));
  return stage_adjoint_planes(m, lim, dt, rk, stage, dtime, 0, -1, 0, -1, c_begin, c_end, x, mu,
                              lam_a, lam_b, out, u_f, w_f, stream);
}

fl_status fl_adjoint_workspace_size(const fl_mesh *m, fl_dtype dt, int rk, int64_t nsteps,
                                    int64_t every, size_t *bytes) {
  if (m == nullptr || bytes == nullptr) return fail(FL_EINVAL, "NULL argument");
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (dt != FL_F32 && dt != FL_F64) return fail(FL_EINVAL, "unknown dtype");
  if (nsteps < 0 || every < 1) return fail(FL_EINVAL, "nsteps >= 0 and checkpoint_every >= 1");
  *bytes = adjoint_ws_bytes(m, dt, rk, nsteps, every);
  return FL_OK;
}

}  // extern "C"

namespace {

// Everything the two checkpointed entry points share: argument checks and
// the workspace layout [checkpoints | segment stage states | 3 adjoints].
struct Sweep {
  const fl_mesh *m;
  int lim;
  fl_dtype dt;
  int rk, S;
  double dtime;
  int64_t nsteps, every, nck;
  size_t one, bytes;
  char *base;
  const void *u;
  cudaStream_t st;
  void *ck(int64_t i) const { return base + one * i; }
  void *slot(int64_t i) const { return base + one * (nck + i); }
  void *lam(int i) const { return base + one * (nck + S * every + 1 + i); }
  // w_f = dt (A/V) u_f when dt > 0 (the forward stages fold their flux
  // product with it and the adjoint stages take b instead of b dt), else
  // (A/V) u_f for the adjoint stages only
  void *cu() const { return base + one * (nck + S * every + 1 + 3); }
  bool cu_dt() const { return dtime > 0; }
  // branch codes of stage i = S n + s of the segment (FP64 pre-scaled
  // stages of the piecewise-linear limiters: the adjoint reads them instead
  // of recomputing the forward stage's differences)
  bool use_codes() const {
    return m->kind == 0 && dt == FL_F64 && cu_dt() && lim != LIM_VANLEER;
  }
  unsigned char *codes(int64_t i) const {
    return reinterpret_cast<unsigned char *>(base + one * (nck + S * every + 1 + 3) +
                                             align256((size_t)m->F * dsize(dt))) +
           (size_t)m->F * i;
  }
  cudaError_t prescale() const {
    // structured: (fac / h_axis) u_f; face-based: fac A_f u_f
    return m->kind == 1 ? unstruct_scale_area(m, dt, u, cu(), cu_dt() ? dtime : 1.0, st)
                        : struct_scale_faces(m, dt, u, cu(), cu_dt() ? dtime : 1.0, st);
  }
  cudaError_t stage(const void *x, const void *thn, void *y, int seed, double a, double b,
                    void *code_out = nullptr) const {
    StageArgs s;
    s.x = x; s.thn = thn; s.y = y; s.u = u; s.dt = dtime; s.seed = seed; s.a = a; s.b = b;
    if (cu_dt()) s.w = cu();
    s.codes = code_out;
    return m->kind == 1 ? unstruct_stage(m, lim, dt, s, st) : struct_stage(m, lim, dt, s, st);
  }
  // one forward step from slot(S n) storing its stage inputs (and, when
  // `codes_on`, their branch codes); the result lands in slot(S (n + 1))
  cudaError_t fwd_step(int64_t n, bool codes_on = false) const {
    auto cd = [&](int64_t i) -> void * { return codes_on ? codes(i) : nullptr; };
    if (S == 1) return stage(slot(n), slot(n), slot(n + 1), 0, 0.0, 1.0, cd(n));
    cudaError_t r = stage(slot(3 * n), slot(3 * n), slot(3 * n + 1), 0, 0.0, 1.0, cd(3 * n));
    if (r == cudaSuccess)
      r = stage(slot(3 * n + 1), slot(3 * n), slot(3 * n + 2), 1, 0.75, 0.25, cd(3 * n + 1));
    if (r == cudaSuccess)
      r = stage(slot(3 * n + 2), slot(3 * n), slot(3 * n + 3), 1, 1.0 / 3.0, 2.0 / 3.0,
                cd(3 * n + 2));
    return r;
  }
};

fl_status sweep_setup(Sweep &w, const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                      int64_t nsteps, int64_t every, const void *u_f, void *ws, size_t ws_bytes,
                      void *stream) {
  FL_TRY(check_mesh(m));
  FL_TRY(check_enums(lim, dt));
  if (rk != 1 && rk != 3) return fail(FL_EINVAL, "rk_order must be 1 or 3");
  if (nsteps < 0 || every < 1) return fail(FL_EINVAL, "nsteps >= 0 and checkpoint_every >= 1");
  if (!std::isfinite(dtime)) return fail(FL_EINVAL, "dt is not finite");
  if (m->kind == 1) FL_TRY(unstruct_adjoint_prepare(m));
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(u_f, m->F * es, "u_f"));
  const size_t need = adjoint_ws_bytes(m, dt, rk, nsteps, every);
  if (ws_bytes < need) return fail(FL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return fail(FL_EINVAL, "workspace must be 256-byte aligned");
  FL_TRY(check_buffer(ws, need, "workspace"));
  w.m = m;
  w.lim = lim;
  w.dt = dt;
  w.rk = rk;
  w.S = (rk == 3) ? 3 : 1;
  w.dtime = dtime;
  w.nsteps = nsteps;
  w.every = every;
  w.nck = (nsteps + every - 1) / every;
  w.one = align256((size_t)m->C * es);
  w.bytes = (size_t)m->C * es;
  w.base = static_cast<char *>(ws);
  w.u = u_f;
  w.st = as_stream(stream);
  return FL_OK;
}

// forward rollout in the segment slots, copying theta to checkpoint c at
// every multiple of `every`; theta0 in, theta_T out (may alias)
cudaError_t sweep_forward(const Sweep &w, const void *theta0, void *thetaT) {
  cudaError_t e = w.prescale();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.slot(0), theta0, w.bytes, cudaMemcpyDeviceToDevice, w.st);
  for (int64_t n = 0; n < w.nsteps && e == cudaSuccess; ++n) {
    if (n % w.every == 0)
      e = cudaMemcpyAsync(w.ck(n / w.every), w.slot(0), w.bytes, cudaMemcpyDeviceToDevice, w.st);
    if (e == cudaSuccess) e = w.fwd_step(0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.slot(0), w.slot(w.S), w.bytes, cudaMemcpyDeviceToDevice, w.st);
  }
  if (e == cudaSuccess && thetaT != nullptr)
    e = cudaMemcpyAsync(thetaT, w.slot(0), w.bytes, cudaMemcpyDeviceToDevice, w.st);
  return e;
}

// reverse sweep from the checkpoints: lambda_T in, lambda_0 out
cudaError_t sweep_reverse(const Sweep &w, const void *lambda_T, void *lambda_0) {
  void *lam = w.lam(0), *la = w.lam(1), *lbb = w.lam(2);
  cudaError_t e = cudaMemcpyAsync(lam, lambda_T, w.bytes, cudaMemcpyDeviceToDevice, w.st);
  if (e == cudaSuccess) e = w.prescale();
  for (int64_t c = w.nck - 1; c >= 0 && e == cudaSuccess; --c) {
    const int64_t len = std::min<int64_t>(w.every, w.nsteps - c * w.every);
    e = cudaMemcpyAsync(w.slot(0), w.ck(c), w.bytes, cudaMemcpyDeviceToDevice, w.st);
    const bool codes = w.use_codes();
    for (int64_t n = 0; n < len && e == cudaSuccess; ++n) e = w.fwd_step(n, codes);
    auto cd = [&](int64_t i) -> const void * { return codes ? w.codes(i) : nullptr; };
    for (int64_t n = len - 1; n >= 0 && e == cudaSuccess; --n) {
      AdjArgs a;
      a.u = w.u;
      a.cu = w.cu();
      a.cu_dt = w.cu_dt();
      a.dt = w.dtime;
      if (w.S == 1) {
        // lam' = lam + dt R'(x)^T lam
        a.x = w.slot(n); a.mu = lam; a.out = la; a.b = 1.0; a.codes = cd(n);
        e = adjoint_any(w.m, w.lim, w.dt, a, w.st);
        void *t = lam;
        lam = la;
        la = t;
      } else {
        // stage 3: la = 2/3 (lam + dt R'(x2)^T lam)
        a.x = w.slot(3 * n + 2); a.mu = lam; a.out = la; a.b = 2.0 / 3.0; a.codes = cd(3 * n + 2);
        e = adjoint_any(w.m, w.lim, w.dt, a, w.st);
        if (e != cudaSuccess) break;
        // stage 2: lbb = 1/4 (la + dt R'(x1)^T la)
        a.x = w.slot(3 * n + 1); a.mu = la; a.out = lbb; a.b = 0.25; a.codes = cd(3 * n + 1);
        e = adjoint_any(w.m, w.lim, w.dt, a, w.st);
        if (e != cudaSuccess) break;
        // stage 1: lam = 1/3 lam + 3/4 la + (lbb + dt R'(x0)^T lbb)
        a.x = w.slot(3 * n); a.mu = lbb; a.out = lam; a.b = 1.0; a.codes = cd(3 * n);
        // e1: the forward stage 3's weight of thn, as the forward kernels used it
        a.v1 = lam; a.v2 = la; a.e2 = 0.75;
        a.e1 = w.dt == FL_F64 ? blend_a<double>(1.0 / 3.0, 2.0 / 3.0)
                              : (double)blend_a<float>(1.0 / 3.0, 2.0 / 3.0);
        e = adjoint_any(w.m, w.lim, w.dt, a, w.st);
      }
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(lambda_0, lam, w.bytes, cudaMemcpyDeviceToDevice, w.st);
  return e;
}

}  // namespace

extern "C" {

fl_status fl_step_rk_checkpointed(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk,
                                  double dtime, int64_t nsteps, int64_t every, void *theta,
                                  const void *u_f, void *ws, size_t ws_bytes, void *stream) {
  Sweep w;
  FL_TRY(sweep_setup(w, m, lim, dt, rk, dtime, nsteps, every, u_f, ws, ws_bytes, stream));
  FL_TRY(check_buffer(theta, m->C * dsize(dt), "theta"));
  if (m->C == 0 || nsteps == 0) return FL_OK;
  cudaError_t e = sweep_forward(w, theta, theta);
  if (e != cudaSuccess) return cuda_fail(e, "checkpointed forward");
  return FL_OK;
}

fl_status fl_step_rk_adjoint_from_checkpoints(const fl_mesh *m, fl_limiter lim, fl_dtype dt,
                                              int rk, double dtime, int64_t nsteps, int64_t every,
                                              const void *u_f, const void *lambda_T,
                                              void *lambda_0, void *ws, size_t ws_bytes,
                                              void *stream) {
  Sweep w;
  FL_TRY(sweep_setup(w, m, lim, dt, rk, dtime, nsteps, every, u_f, ws, ws_bytes, stream));
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(lambda_T, m->C * es, "lambda_T"));
  FL_TRY(check_buffer(lambda_0, m->C * es, "lambda_0"));
  if (m->C == 0) return FL_OK;
  cudaError_t e = (nsteps == 0)
                      ? cudaMemcpyAsync(lambda_0, lambda_T, w.bytes, cudaMemcpyDeviceToDevice, w.st)
                      : sweep_reverse(w, lambda_T, lambda_0);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint sweep");
  return FL_OK;
}

fl_status fl_step_rk_adjoint(const fl_mesh *m, fl_limiter lim, fl_dtype dt, int rk, double dtime,
                             int64_t nsteps, int64_t every, const void *theta0, const void *u_f,
                             const void *lambda_T, void *lambda_0, void *ws, size_t ws_bytes,
                             void *stream) {
  Sweep w;
  FL_TRY(sweep_setup(w, m, lim, dt, rk, dtime, nsteps, every, u_f, ws, ws_bytes, stream));
  const size_t es = dsize(dt);
  FL_TRY(check_buffer(theta0, m->C * es, "theta0"));
  FL_TRY(check_buffer(lambda_T, m->C * es, "lambda_T"));
  FL_TRY(check_buffer(lambda_0, m->C * es, "lambda_0"));
  if (m->C == 0) return FL_OK;
  cudaError_t e = cudaSuccess;
  if (nsteps == 0) {
    e = cudaMemcpyAsync(lambda_0, lambda_T, w.bytes, cudaMemcpyDeviceToDevice, w.st);
  } else {
    e = sweep_forward(w, theta0, nullptr);
    if (e == cudaSuccess) e = sweep_reverse(w, lambda_T, lambda_0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint sweep");
  return FL_OK;
}

}  // extern "C"
