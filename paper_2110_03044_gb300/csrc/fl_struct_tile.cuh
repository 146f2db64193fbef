// fl_struct_tile.cuh -- one tile of the fused limited-convection stage on a
// periodic Cartesian mesh (see fl_structured.cu for the method), shared by
// the single-mesh kernel and the persistent batched kernel.
#pragma once

#include <cuda_runtime.h>

#include "fl_face.cuh"

namespace fl {
namespace {

constexpr int TX = 32;  // one warp along x

template <class T>
struct SParams {
  const T *x;      // stage input theta (neighbour reads)
  const T *thn;    // theta^n (own cell only; may alias y)
  T *y;            // output: stage result or R (own cell only)
  T *thf;          // optional face values (apply mode), may be null
  const T *u;      // face velocities
  int nx, ny, nz;
  int act_x, act_y, act_z;
  long long ux_off, uy_off, uz_off;
  long long plane;  // nx*ny
  T cx, cy, cz;     // multiply (phi_minus - phi_plus) of each axis
  T a, b;           // seed = a*thn + b*x  (COMBINE) or x (PLAIN) or 0 (APPLY)
  T g;              // MOD: velocity factor of the stage (see stage_tile)
  unsigned long long flip;  // sign mask toggled into u before the upwind test (g < 0)
  unsigned char *codes;     // CODES: branch code per face (layout of u), or null
  int tiles_x, tiles_y, zchunk;
  // the tiles cover planes [zlo, min(zhi, nz)) (a plane range of a
  // decomposed mesh; the whole mesh by default)
  int zlo = 0, zhi = 1 << 30;
  int ylo = 0, yhi = 1 << 30;  // and rows [ylo, min(yhi, ny)) of them
  // padded copy of a batched box (fl_struct_pad4.cuh): row pitch (0 for
  // the box's own layout) and the ghost rows / planes before the first
  int pitch = 0, gy = 0, gz = 0;
};

enum { SEED_PLAIN = 0, SEED_COMBINE = 1, SEED_APPLY = 2 };

// FP64 cell differences: 1 forms the exact ones on the integer pipe
// (FT<double>::sub_exact), 0 takes the FP64 subtraction for all
#ifndef FL_SUB_INT
#define FL_SUB_INT 0
#endif
template <class T>
__device__ __forceinline__ T cell_diff(T a, T b) {
  if constexpr (FL_SUB_INT && sizeof(T) == 8) return FT<T>::sub_exact(a, b);
  else return FT<T>::sub(a, b);
}

// Keeps a value as computed: the compiler may no longer recompute it from
// its operands at a later use.  Under the register cap it otherwise
// rematerialised the z-window differences, spending FP64 pipe slots.
__device__ __forceinline__ void keep(double &x) { asm("" : "+d"(x)); }
__device__ __forceinline__ void keep(float &x) { asm("" : "+f"(x)); }

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// PRE: p.u holds w_f = dt (A/V) u_f (pre-scaled once per call, same sign as
// u_f) and p.cx/cy/cz are unused.  Each face then keeps theta_f instead of
// its flux, and a cell adds w theta_f of its six faces with one fma each:
// the flux product is folded into the cell update (12 FP64 operations per
// cell and stage instead of 15).  The two cells of a face use the same w and
// theta_f, so the update stays conservative to rounding.  s_ux / s_uy are
// then read by the cell update too and are double-buffered by plane parity.
//
// A stage whose velocity is g u_f (a time-modulated flow) toggles the sign of
// every u before its upwind test when g < 0 (p.flip).  Without PRE, g is part
// of p.cx/cy/cz; with PRE and MOD the six w theta_f terms are summed first
// and added as x + g S.
//
// CODES: the tile also writes, for every face it owns, the branch code of
// its limited value (lin_code, bit 3 = s > 0), which the adjoint of the same
// stage reads instead of recomputing theta's differences.
template <class T, int LIM, int SEED, int TY, bool PRE = false, bool MOD = false,
          bool CODES = false>
__device__ __forceinline__ void stage_tile(const SParams<T> &p, int tile) {
  using F = FT<T>;
  constexpr int NT = TX * TY;
  constexpr int SW = TX + 4;  // s_th row pitch
  constexpr int NUB = PRE ? 2 : 1;
  // FP32 stage updates keep each face's flux u theta_f, taken on the native
  // FP32 min/max with its sign on the FMA pipe (native_flux): the FP32 ALU
  // pipe, not the FP64 one, bounds them, and the integer-domain limiter made
  // for FP64 costs it more instructions
  constexpr bool NATIVE = sizeof(T) == 4 && !PRE && SEED != SEED_APPLY && !CODES;
  __shared__ T s_th[(TY + 4) * SW];
  __shared__ T s_dx[TY * (TX + 3)];
  __shared__ T s_dy[(TY + 3) * TX];
  __shared__ T s_fx[TY * (TX + 1)];
  __shared__ T s_fy[(TY + 1) * TX];
  __shared__ T s_uxb[NUB][TY * (TX + 1)];  // u of x faces m = x0-1 .. x0+TX-1
  __shared__ T s_uyb[NUB][(TY + 1) * TX];  // u of y faces m = y0-1 .. y0+TY-1
  __shared__ int s_wx[TX + 4];
  __shared__ int s_wy[TY + 4];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  int bid = tile;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = p.ylo + by * TY;
  const int z0 = p.zlo + bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, min(p.nz, p.zhi));
  const int nx = p.nx, ny = p.ny, nz = p.nz;

  // wrapped coordinates of the tile's columns/rows, halo included:
  // s_wx[w] = (x0 - 2 + w) mod nx, s_wy[w] = (y0 - 2 + w) mod ny
  if (tid < TX + 4) s_wx[tid] = wrap(x0 - 2 + tid, nx);
  if (tid < TY + 4) s_wy[tid] = wrap(y0 - 2 + tid, ny);
  __syncthreads();

  const bool valid = (x0 + tx < nx) && (y0 + ty < min(ny, p.yhi));
  // Addressing: one 64-bit base pointer per stream and 32-bit element
  // offsets (every cell or plane offset is below n_cells < 2^31), so that a
  // load costs one wide multiply-add rather than 64-bit index arithmetic
  const unsigned plane = (unsigned)p.plane;
  const unsigned col = (unsigned)s_wx[tx + 2] + (unsigned)nx * (unsigned)s_wy[ty + 2];
  const T *__restrict__ Ux = p.u + p.ux_off;
  const T *__restrict__ Uy = p.u + p.uy_off;
  const T *__restrict__ Uz = p.u + p.uz_off;
  const bool need_x = p.act_x, need_y = p.act_y, need_z = p.act_z;

  // halo cells of s_th: 2 columns left/right of every row, 2 rows above/below
  constexpr int NH = 4 * (TX + TY);
  static_assert(NH <= NT, "halo items exceed threads");
  int h_slot = -1;
  unsigned h_off = 0;
  if (tid < 4 * TY) {  // x halo
    const int r = tid >> 2, k4 = tid & 3;
    const int c = (k4 < 2) ? k4 : (TX + k4);  // 0,1,TX+2,TX+3
    h_slot = (r + 2) * SW + c;
    h_off = (unsigned)s_wx[c] + (unsigned)nx * (unsigned)s_wy[r + 2];
  } else if (tid < NH) {  // y halo
    const int t = tid - 4 * TY;
    const int k4 = t / TX, c = t % TX;
    const int r = (k4 < 2) ? k4 : (TY + k4);  // 0,1,TY+2,TY+3
    h_slot = r * SW + c + 2;
    h_off = (unsigned)s_wx[c + 2] + (unsigned)nx * (unsigned)s_wy[r];
  }
  // halo faces: the -x face of every row (x0-1) and the -y face of every
  // column (y0-1); each thread owns the +x, +y and +z faces of its cell
  int hu_slot = -1;
  unsigned hu_off = 0;
  const T *hu_base = Ux;
  bool hu_is_x = false;
  if (tid < TY) {
    if (need_x) {
      hu_slot = tid * (TX + 1);
      hu_off = (unsigned)s_wx[1] + (unsigned)nx * (unsigned)s_wy[tid + 2];
      hu_is_x = true;
    }
  } else if (tid < TY + TX) {
    if (need_y) {
      const int c = tid - TY;
      hu_slot = c;
      hu_base = Uy;
      hu_off = (unsigned)s_wx[c + 2] + (unsigned)nx * (unsigned)s_wy[1];
    }
  }

  // ---- plane loads, software-pipelined one plane ahead
  struct Plane {
    T ux, uy, uz, thn, h, hu;
  };
  auto load_plane = [&](int k, Plane &q) {
    const unsigned pk = plane * (unsigned)k;
    if (need_x) q.ux = Ux[col + pk];
    if (need_y) q.uy = Uy[col + pk];
    if (need_z) q.uz = Uz[col + pk];
    if (SEED == SEED_COMBINE) q.thn = p.thn[col + pk];
    if (h_slot >= 0) q.h = p.x[h_off + pk];
    if (hu_slot >= 0) q.hu = hu_base[hu_off + pk];
  };
  Plane cur{}, nxt{};

  // ---- z prologue: columns k-2 .. k+1 around z0, and the flux of face z0-1/2
  T th0, thp1, thp2 = T(0), dz_m1 = T(0), dz_0 = T(0), fz_prev = T(0), wz_prev = T(0);
  if (need_z) {
    const T tm2 = p.x[col + plane * (unsigned)wrap(z0 - 2, nz)];
    const T tm1 = p.x[col + plane * (unsigned)wrap(z0 - 1, nz)];
    th0 = p.x[col + plane * (unsigned)z0];
    thp1 = p.x[col + plane * (unsigned)wrap(z0 + 1, nz)];
    thp2 = p.x[col + plane * (unsigned)wrap(z0 + 2, nz)];
    const T d_m2 = F::sub(tm1, tm2);
    dz_m1 = F::sub(th0, tm1);
    dz_0 = F::sub(thp1, th0);
    keep(dz_m1);
    keep(dz_0);
    const T uz = Uz[col + plane * (unsigned)wrap(z0 - 1, nz)];
    const bool sp = upwind_positive(sign_toggled(uz, p.flip));
    // (the same value the previous z chunk computes for this face)
    if constexpr (NATIVE) {
      fz_prev = native_flux<LIM>(uz, sp ? tm1 : th0, dz_m1, sp ? d_m2 : dz_0, (unsigned)p.flip);
    } else {
      const T thf = limited_face<T, LIM>(sp ? tm1 : th0, dz_m1, sp ? d_m2 : dz_0, sp);
      fz_prev = PRE ? thf : face_flux(uz, thf);
    }
    wz_prev = uz;
  } else {
    th0 = p.x[col];
    thp1 = th0;
  }
  load_plane(z0, cur);

  for (int k = z0; k < z1; ++k) {
    const unsigned pk = plane * (unsigned)k;
    T *s_ux = s_uxb[PRE ? (k & 1) : 0];
    T *s_uy = s_uyb[PRE ? (k & 1) : 0];
    // -------------------------------------------- fill plane k
    s_th[(ty + 2) * SW + tx + 2] = th0;
    if (h_slot >= 0) s_th[h_slot] = cur.h;
    if (need_x) s_ux[ty * (TX + 1) + tx + 1] = cur.ux;
    if (need_y) s_uy[(ty + 1) * TX + tx] = cur.uy;
    if (hu_slot >= 0) {
      if (hu_is_x) s_ux[hu_slot] = cur.hu;
      else s_uy[hu_slot] = cur.hu;
    }
    // -------------------------------------- prefetch plane k + 1
    T tp3 = T(0);
    if (k + 1 < z1) {
      load_plane(k + 1, nxt);
      if (need_z) tp3 = p.x[col + plane * (unsigned)wrap(k + 3, nz)];
    }
    __syncthreads();
    // ------------------------------------------- phase A: differences
    if (need_x) {
      for (int it = tid; it < TY * (TX + 3); it += NT) {
        const int r = it / (TX + 3), q = it - r * (TX + 3);
        const T *row = &s_th[(r + 2) * SW];
        s_dx[it] = cell_diff<T>(row[q + 1], row[q]);
      }
    }
    if (need_y) {
      for (int it = tid; it < (TY + 3) * TX; it += NT) {
        const int r = it / TX, c = it - r * TX;
        s_dy[it] = cell_diff<T>(s_th[(r + 1) * SW + c + 2], s_th[r * SW + c + 2]);
      }
    }
    T dz_p1 = T(0);
    if (need_z) {
#if FL_SUB_INT >= 2
      dz_p1 = cell_diff<T>(thp2, thp1);
#else
      dz_p1 = F::sub(thp2, thp1);
#endif
      keep(dz_p1);
    }
    __syncthreads();
    // ----------------------------------------------- phase B: fluxes
    if (need_x) {
      for (int it = tid; it < TY * (TX + 1); it += NT) {
        const int r = it / (TX + 1), q = it - r * (TX + 1);  // face m = x0-1+q
        const T uf = s_ux[it];
        const bool sp = upwind_positive(sign_toggled(uf, p.flip));
        const T *dr = &s_dx[r * (TX + 3)];
        const T *tr = &s_th[(r + 2) * SW];
        if constexpr (NATIVE) {
          s_fx[it] = native_flux<LIM>(uf, sp ? tr[q + 1] : tr[q + 2], dr[q + 1],
                                      sp ? dr[q] : dr[q + 2], (unsigned)p.flip);
          continue;
        }
        const T thf = limited_face<T, LIM>(sp ? tr[q + 1] : tr[q + 2], dr[q + 1],
                                           sp ? dr[q] : dr[q + 2], sp);
        s_fx[it] = PRE ? thf : face_flux(uf, thf);
        if (CODES && q >= 1 && x0 + q - 1 < nx && y0 + r < ny)
          p.codes[p.ux_off + (s_wx[q + 1] + (unsigned)nx * (unsigned)s_wy[r + 2] + pk)] =
              (unsigned char)(lin_code<T, LIM>(dr[q + 1], sp ? dr[q] : dr[q + 2]) | (sp ? 8 : 0));
        if (SEED == SEED_APPLY && p.thf != nullptr) {
          if (q >= 1 && x0 + q - 1 < nx && y0 + r < ny)
            p.thf[p.ux_off + (s_wx[q + 1] + (unsigned)nx * (unsigned)s_wy[r + 2] + pk)] = thf;
        }
      }
    }
    if (need_y) {
      for (int it = tid; it < (TY + 1) * TX; it += NT) {
        const int r = it / TX, c = it - r * TX;  // face m = y0-1+r
        const T uf = s_uy[it];
        const bool sp = upwind_positive(sign_toggled(uf, p.flip));
        if constexpr (NATIVE) {
          s_fy[it] = native_flux<LIM>(
              uf, sp ? s_th[(r + 1) * SW + c + 2] : s_th[(r + 2) * SW + c + 2],
              s_dy[(r + 1) * TX + c], sp ? s_dy[r * TX + c] : s_dy[(r + 2) * TX + c],
              (unsigned)p.flip);
          continue;
        }
        const T thf = limited_face<T, LIM>(
            sp ? s_th[(r + 1) * SW + c + 2] : s_th[(r + 2) * SW + c + 2], s_dy[(r + 1) * TX + c],
            sp ? s_dy[r * TX + c] : s_dy[(r + 2) * TX + c], sp);
        s_fy[it] = PRE ? thf : face_flux(uf, thf);
        if (CODES && r >= 1 && x0 + c < nx && y0 + r - 1 < ny)
          p.codes[p.uy_off + (s_wx[c + 2] + (unsigned)nx * (unsigned)s_wy[r + 1] + pk)] = (unsigned char)(
              lin_code<T, LIM>(s_dy[(r + 1) * TX + c], sp ? s_dy[r * TX + c] : s_dy[(r + 2) * TX + c]) |
              (sp ? 8 : 0));
        if (SEED == SEED_APPLY && p.thf != nullptr) {
          if (r >= 1 && x0 + c < nx && y0 + r - 1 < ny)
            p.thf[p.uy_off + (s_wx[c + 2] + (unsigned)nx * (unsigned)s_wy[r + 1] + pk)] = thf;
        }
      }
    }
    T fz = T(0);
    if (need_z) {
      const bool sp = upwind_positive(sign_toggled(cur.uz, p.flip));
      T thf = T(0);
      if constexpr (NATIVE) {
        fz = native_flux<LIM>(cur.uz, sp ? th0 : thp1, dz_0, sp ? dz_m1 : dz_p1,
                              (unsigned)p.flip);
      } else {
        thf = limited_face<T, LIM>(sp ? th0 : thp1, dz_0, sp ? dz_m1 : dz_p1, sp);
        fz = PRE ? thf : face_flux(cur.uz, thf);
      }
      if (CODES && valid)
        p.codes[p.uz_off + (col + pk)] =
            (unsigned char)(lin_code<T, LIM>(dz_0, sp ? dz_m1 : dz_p1) | (sp ? 8 : 0));
      if (SEED == SEED_APPLY && p.thf != nullptr && valid) p.thf[p.uz_off + (col + pk)] = thf;
    }
    __syncthreads();
    // ------------------------------------------------ phase C: update
    if (PRE && valid) {
      // y = x + sum (w theta_f)_minus - (w theta_f)_plus, then the RK blend
      T acc = MOD ? T(0) : th0;
      if (need_x) {
        const int i = ty * (TX + 1) + tx;
        acc = F::fma(-s_ux[i + 1], s_fx[i + 1], acc);
        acc = F::fma(s_ux[i], s_fx[i], acc);
      }
      if (need_y) {
        acc = F::fma(-s_uy[(ty + 1) * TX + tx], s_fy[(ty + 1) * TX + tx], acc);
        acc = F::fma(s_uy[ty * TX + tx], s_fy[ty * TX + tx], acc);
      }
      if (need_z) {
        acc = F::fma(-cur.uz, fz, acc);
        acc = F::fma(wz_prev, fz_prev, acc);
      }
      if (MOD) acc = F::fma(p.g, acc, th0);
      if (SEED == SEED_COMBINE) acc = F::fma(p.b, acc, F::mul(p.a, cur.thn));
      p.y[col + pk] = acc;
    } else if (valid) {
      T acc;
      if (SEED == SEED_PLAIN) acc = th0;
      else if (SEED == SEED_COMBINE) acc = F::fma(p.a, cur.thn, F::mul(p.b, th0));
      else acc = T(0);
      if (need_x) {
        acc = F::fma(-p.cx, s_fx[ty * (TX + 1) + tx + 1], acc);
        acc = F::fma(p.cx, s_fx[ty * (TX + 1) + tx], acc);
      }
      if (need_y) {
        acc = F::fma(-p.cy, s_fy[(ty + 1) * TX + tx], acc);
        acc = F::fma(p.cy, s_fy[ty * TX + tx], acc);
      }
      if (need_z) {
        acc = F::fma(-p.cz, fz, acc);
        acc = F::fma(p.cz, fz_prev, acc);
      }
      p.y[col + pk] = acc;
    }
    // --------------------------------------------------------- rotate
    if (need_z) wz_prev = cur.uz;
    cur = nxt;
    if (need_z) {
      fz_prev = fz;
      dz_m1 = dz_0;
      dz_0 = dz_p1;
      th0 = thp1;
      thp1 = thp2;
      thp2 = tp3;
    } else if (k + 1 < z1) {
      th0 = p.x[col + plane * (unsigned)(k + 1)];
    }
  }
}


}  // namespace
}  // namespace fl
