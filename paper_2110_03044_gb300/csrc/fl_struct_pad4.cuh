// fl_struct_pad4.cuh -- FP32 stage tile for the batched persistent kernel
// (fl_batch.cu) on boxes copied into a padded layout with periodic ghost
// cells.
//
// The method, the face arithmetic and the order of the cell sums are those
// of the other FP32 tiles (fl_struct_tma.cu, fl_struct_reg.cuh,
// fl_struct_flat.cuh: Valle et al., Algorithm 4 with Algorithm 1's limited
// face values on Sweby's Cartesian stencil; x, y, z, the + face before the -
// face), so all of them give the same bits.
//
// The boxes of a batch have any nx, so in their own layout a thread's cells
// are not 16-byte aligned and rows end anywhere in a warp's run.  For the
// whole of a call the batch keeps each box with nx >= 8 in a padded copy:
//   * a row holds P = round_up(nx + 4, 4) cells: two ghost columns (x = -2,
//     -1), the nx cells at columns 2 .. nx + 1, and at least two ghost
//     columns (x = nx, nx + 1) after them;
//   * two ghost rows before and after the ny rows (when ny > 1), two ghost
//     planes before and after the nz planes (when nz > 1);
//   * a ghost cell holds the periodic image of a cell; the copy in fills them
//     all, and every stage writes the images its stencil reads (x = -2, -1,
//     nx, nx + 1 of the box's rows, y = -2, -1, ny, ny + 1 and z = -2, -1,
//     nz, nz + 1 of the box's cells) together with the cells themselves.
// In this layout the stage has no periodic wrap to handle:
//   * a warp owns a run of 128 consecutive cells of the ny rows of a plane
//     (ghost columns included), lane l four consecutive cells of one row,
//     16-byte aligned: every array is read with one 16-byte copy per lane
//     and plane (cp.async into shared memory, a plane ahead), the y
//     neighbours at -2P .. +2P, the z window in registers;
//   * the x window (cells -2 .. 5 from the first) comes from the lane's own
//     four cells and two shuffled from each neighbouring lane, lanes 0 and
//     31 copying their outer pair; each lane evaluates its five x faces
//     (-1 .. 3), so no flux crosses lanes and no lane evaluates a face
//     alone while the others wait;
//   * lanes on ghost columns compute and store nothing of theirs.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "fl_face.cuh"
#include "fl_struct_reg.cuh"
#include "fl_struct_tile.cuh"

namespace fl {
namespace {

constexpr int PAD_RUN = 128;  // cells of one warp's run: 32 lanes x 4
constexpr int PAD_GX = 2;     // ghost columns before a row's first cell

// Geometry of a box's padded copy.
struct PadGeom {
  int P, PY, PZ, gy, gz;
  long long plane, vol;
};
__host__ __device__ inline PadGeom pad_geom(int nx, int ny, int nz) {
  PadGeom g;
  g.P = (nx + 4 + 3) / 4 * 4;
  g.gy = ny > 1 ? 2 : 0;
  g.gz = nz > 1 ? 2 : 0;
  g.PY = ny + 2 * g.gy;
  g.PZ = nz + 2 * g.gz;
  g.plane = (long long)g.P * g.PY;
  g.vol = g.plane * g.PZ;
  return g;
}

__device__ __forceinline__ float4 ldf4(const float *a, unsigned o) {
  return *reinterpret_cast<const float4 *>(a + o);
}
__device__ __forceinline__ void stf4(float *a, unsigned o, float4 v) {
  *reinterpret_cast<float4 *>(a + o) = v;
}

// 16-byte values a thread stages per plane (see stage_pad4), and the stride
// of a thread's staging block: two slots of PAD_NA values plus one, so that
// the 128-bit reads of eight consecutive threads fall in distinct banks
constexpr int PAD_NA = 11;
constexpr int PAD_STRIDE = 2 * PAD_NA + 1;
constexpr int PAD_STAGE_BYTES = PAD_STRIDE * 16;

// cp.async of `bytes` (16, 8 or 4) into shared address d + OFF
template <int OFF, int BYTES>
__device__ __forceinline__ void cpa(unsigned d, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0+%2], [%1], %3;" ::"r"(d), "l"(src), "n"(OFF),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One work item: run `seg` (of PAD_RUN blockDim.y cells of the ny rows of a
// plane) of every plane in z chunk `zc`.  p holds padded pointers (x, thn,
// y, u with its components p.plane * PZ apart at p.u?_off), p.pitch = P,
// p.plane = P PY, p.gy, p.gz; p.tiles_x runs per plane.  stage: this
// thread's staging block in shared memory (PAD_STRIDE 16-byte values).
//
// The loads of plane k + 1 (the velocities, theta^n, the four y neighbour
// rows, the z-window plane k + 4 and the x halo of lanes 0 and 31) are copied
// into the thread's staging slot with cp.async while plane k is computed, so
// no register holds a load in flight across a plane and their latency hides
// behind a plane's arithmetic.  Each thread reads back only what it copied.
template <int LIM, int SEED>
__device__ __forceinline__ void stage_pad4(const SParams<float> &p, int seg, int zc,
                                           float4 *stage) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr unsigned fl = 0u;  // batched stages run without a velocity factor
  const int lane = threadIdx.x;
  const int nx = p.nx, ny = p.ny, nz = p.nz, P = p.pitch;
  const unsigned PP = (unsigned)p.plane;
  const int rows = ny * P;  // cells of a plane's ny rows
  const int run0 = (seg * (int)blockDim.y + (int)threadIdx.y) * PAD_RUN;
  if (run0 >= rows) return;  // the warp's run lies past the rows
  const bool live = run0 + 4 * lane < rows;
  const int f0 = live ? run0 + 4 * lane : rows - 4;
  const int yrow = f0 / P, c0 = f0 - yrow * P;
  const int xb = c0 - PAD_GX;  // x of the lane's first cell
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, nz);
  const bool need_y = p.act_y, need_z = p.act_z;
  const float *__restrict__ X = p.x;
  const float *__restrict__ Ux = p.u + p.ux_off;
  const float *__restrict__ Uy = p.u + p.uy_off;
  const float *__restrict__ Uz = p.u + p.uz_off;
  float *__restrict__ Y = p.y;
  bool val[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) val[v] = live && xb + v >= 0 && xb + v < nx;
  const bool all4 = val[0] && val[3];
  const unsigned P1 = (unsigned)P, P2 = 2u * (unsigned)P;
  const unsigned ybase = (unsigned)(p.gy * P + f0);
  auto at = [&](int kz) { return (unsigned)(kz + p.gz) * PP + ybase; };
  const bool hal0 = lane == 0 && c0 >= 4, hal31 = lane == 31 && c0 + 4 < P;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(stage);

  // plane j's loads into slot S; the z-window plane j + 3 (with z) or j
  // itself (without z) as value 0
  auto issue_slot = [&](auto slot, int j) {
    constexpr int B = decltype(slot)::value * PAD_NA * 16;
    const unsigned o = at(j);
    if (need_z) {
      if (j + 1 < z1) cpa<B, 16>(sbase, X + (o + 3u * PP));
    } else {
      cpa<B, 16>(sbase, X + o);
    }
    cpa<B + 16, 16>(sbase, Ux + o);
    if (need_z) cpa<B + 32, 16>(sbase, Uz + o);
    if (SEED == SEED_COMBINE) cpa<B + 48, 16>(sbase, p.thn + o);
    if (need_y) {
      cpa<B + 64, 16>(sbase, X + (o - P2));
      cpa<B + 80, 16>(sbase, X + (o - P1));
      cpa<B + 96, 16>(sbase, X + (o + P1));
      cpa<B + 112, 16>(sbase, X + (o + P2));
      cpa<B + 128, 16>(sbase, Uy + o);
      cpa<B + 144, 16>(sbase, Uy + (o - P1));
    }
    if (hal0) {
      cpa<B + 160, 8>(sbase, X + (o - 2u));
      cpa<B + 168, 4>(sbase, Ux + (o - 1u));
    }
    if (hal31) cpa<B + 160, 8>(sbase, X + (o + 4u));
    cpa_commit();
  };
  auto issue = [&](int j, int s) {
    if (s == 0) issue_slot(std::integral_constant<int, 0>(), j);
    else issue_slot(std::integral_constant<int, 1>(), j);
  };

  // ------------------------------------------------ z window
  float th0[4], thp1[4], thp2[4], dzm[4], dz0[4], fzp[4];
  {
    const float4 c = ldf4(X, at(z0));
    th0[0] = c.x, th0[1] = c.y, th0[2] = c.z, th0[3] = c.w;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) thp1[v] = thp2[v] = dzm[v] = dz0[v] = fzp[v] = 0.f;
  issue(z0, 0);
  if (need_z) {
    const float4 m2 = ldf4(X, at(z0 - 2)), m1 = ldf4(X, at(z0 - 1));
    const float4 p1 = ldf4(X, at(z0 + 1)), p2 = ldf4(X, at(z0 + 2));
    const float4 um = ldf4(Uz, at(z0 - 1));
    const float tm2[4] = {m2.x, m2.y, m2.z, m2.w}, tm1[4] = {m1.x, m1.y, m1.z, m1.w};
    const float tp1[4] = {p1.x, p1.y, p1.z, p1.w}, tp2[4] = {p2.x, p2.y, p2.z, p2.w};
    const float uzm[4] = {um.x, um.y, um.z, um.w};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      thp1[v] = tp1[v];
      thp2[v] = tp2[v];
      const float d_m2 = __fsub_rn(tm1[v], tm2[v]);
      dzm[v] = __fsub_rn(th0[v], tm1[v]);
      dz0[v] = __fsub_rn(thp1[v], th0[v]);
      fzp[v] = reg_flux<LIM>(uzm[v], tm1[v], th0[v], dzm[v], d_m2, dz0[v], fl);
    }
  }

  for (int k = z0; k < z1; ++k) {
    const unsigned o = at(k);
    const int s = (k - z0) & 1;
    if (k + 1 < z1) issue(k + 1, s ^ 1);
    else cpa_commit();
    cpa_wait1();  // plane k's copies have landed
    const float4 *d = stage + s * PAD_NA;
    if (!need_z) {
      const float4 c = d[0];
      th0[0] = c.x, th0[1] = c.y, th0[2] = c.z, th0[3] = c.w;
    }
    // the plane's arithmetic over a face-flux function: first with van
    // Leer's quotient unchecked, flagging a quotient out of its range; a
    // warp that flagged one evaluates the plane again with the checked
    // quotient (both give the checked quotient's bits)
    float acc[4], fz[4], dzp[4];
    auto plane_faces = [&](auto flux) {
      if (SEED == SEED_COMBINE) {
        const float4 tn4 = d[3];
        const float tn[4] = {tn4.x, tn4.y, tn4.z, tn4.w};
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] = __fmaf_rn(p.a, tn[v], __fmul_rn(p.b, th0[v]));
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] = th0[v];
      }
      // ---------------------------------------------- x faces -1 .. 3
      {
        const float4 ux4 = d[1];
        const float *h = reinterpret_cast<const float *>(d + 10);
        float t[8];  // t[j + 2] = theta at position j, j = -2 .. 5
        const float sl2 = __shfl_up_sync(FULL, th0[2], 1), sl1 = __shfl_up_sync(FULL, th0[3], 1);
        const float sr4 = __shfl_down_sync(FULL, th0[0], 1), sr5 = __shfl_down_sync(FULL, th0[1], 1);
        const float su = __shfl_up_sync(FULL, ux4.w, 1);
        t[0] = hal0 ? h[0] : sl2;
        t[1] = hal0 ? h[1] : sl1;
#pragma unroll
        for (int v = 0; v < 4; ++v) t[v + 2] = th0[v];
        t[6] = hal31 ? h[0] : sr4;
        t[7] = hal31 ? h[1] : sr5;
        const float uf[5] = {hal0 ? h[2] : su, ux4.x, ux4.y, ux4.z, ux4.w};
        float dd[7];  // dd[j + 2] = theta(j + 1) - theta(j)
#pragma unroll
        for (int j = 0; j < 7; ++j) dd[j] = __fsub_rn(t[j + 1], t[j]);
        float fx[5];  // fx[m + 1] = flux of face m (between positions m and m + 1)
#pragma unroll
        for (int m = -1; m <= 3; ++m)
          fx[m + 1] = flux(uf[m + 1], t[m + 2], t[m + 3], dd[m + 2], dd[m + 1], dd[m + 3], fl);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[v] = __fmaf_rn(-p.cx, fx[v + 1], acc[v]);
          acc[v] = __fmaf_rn(p.cx, fx[v], acc[v]);
        }
      }
      // ---------------------------------------------- y faces
      if (need_y) {
        const float4 ym2 = d[4], ym1 = d[5], yp1 = d[6], yp2 = d[7];
        const float4 uyp = d[8], uym = d[9];
        const float a2[4] = {ym2.x, ym2.y, ym2.z, ym2.w}, a1[4] = {ym1.x, ym1.y, ym1.z, ym1.w};
        const float b1[4] = {yp1.x, yp1.y, yp1.z, yp1.w}, b2[4] = {yp2.x, yp2.y, yp2.z, yp2.w};
        const float up[4] = {uyp.x, uyp.y, uyp.z, uyp.w}, um[4] = {uym.x, uym.y, uym.z, uym.w};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float t0 = th0[v];
          const float dm2 = __fsub_rn(a1[v], a2[v]), dm1 = __fsub_rn(t0, a1[v]);
          const float d0 = __fsub_rn(b1[v], t0), dp1 = __fsub_rn(b2[v], b1[v]);
          const float fm = flux(um[v], a1[v], t0, dm1, dm2, d0, fl);
          const float fp = flux(up[v], t0, b1[v], d0, dm1, dp1, fl);
          acc[v] = __fmaf_rn(-p.cy, fp, acc[v]);
          acc[v] = __fmaf_rn(p.cy, fm, acc[v]);
        }
      }
      // ---------------------------------------------- z faces
      if (need_z) {
        const float4 uz4 = d[2];
        const float uz[4] = {uz4.x, uz4.y, uz4.z, uz4.w};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          dzp[v] = __fsub_rn(thp2[v], thp1[v]);
          fz[v] = flux(uz[v], th0[v], thp1[v], dz0[v], dzm[v], dzp[v], fl);
          acc[v] = __fmaf_rn(-p.cz, fz[v], acc[v]);
          acc[v] = __fmaf_rn(p.cz, fzp[v], acc[v]);
        }
      }
    };
    if (LIM == LIM_VANLEER) {
      bool far = false;
      plane_faces([&](float u, float cp, float cn, float a, float bp, float bn, unsigned f) {
        return reg_flux_unchecked<LIM>(u, cp, cn, a, bp, bn, f, far);
      });
      if (__any_sync(FULL, far))
        plane_faces([&](float u, float cp, float cn, float a, float bp, float bn, unsigned f) {
          return reg_flux<LIM>(u, cp, cn, a, bp, bn, f);
        });
    } else {
      plane_faces([&](float u, float cp, float cn, float a, float bp, float bn, unsigned f) {
        return reg_flux<LIM>(u, cp, cn, a, bp, bn, f);
      });
    }
    // ---------------------------------------------- store, with the images
    {
      const float4 r = make_float4(acc[0], acc[1], acc[2], acc[3]);
      auto put = [&](unsigned oo) {
        if (all4) {
          stf4(Y, oo, r);
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (val[v]) Y[oo + v] = acc[v];
        }
      };
      put(o);
      if (need_y && yrow < 2) put(o + (unsigned)ny * P1);
      if (need_y && yrow >= ny - 2) put(o - (unsigned)ny * P1);
      if (need_z && k < 2) put(o + (unsigned)nz * PP);
      if (need_z && k >= nz - 2) put(o - (unsigned)nz * PP);
      if (xb < 2 || xb + 3 >= nx - 2) {  // x images of the row's first and last two cells
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (val[v] && xb + v < 2) Y[o + v + nx] = acc[v];
          if (val[v] && xb + v >= nx - 2) Y[o + v - nx] = acc[v];
        }
      }
    }
    // ---------------------------------------------- shift the z window
    if (need_z) {
      float4 pfn = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k + 1 < z1) pfn = d[0];
      const float pv[4] = {pfn.x, pfn.y, pfn.z, pfn.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fzp[v] = fz[v];
        dzm[v] = dz0[v];
        dz0[v] = dzp[v];
        th0[v] = thp1[v];
        thp1[v] = thp2[v];
        thp2[v] = pv[v];
      }
    }
  }
  cpa_wait0();  // nothing of this item stays in flight into the next
}

// The padded copy of box fields (blockIdx.y = box, q = the box's conversion
// parameters: x = its theta, y = the padded theta, u = its face velocities,
// thf = the padded velocities): every padded cell, ghosts included, takes
// the value of its periodic image.  A warp copies a padded row (blocks of
// 32 x 8 threads, eight rows at a time).
__global__ void k_pad_in(const SParams<float> *__restrict__ conv) {
  const SParams<float> q = conv[blockIdx.y];
  if (q.pitch == 0) return;
  const PadGeom g = pad_geom(q.nx, q.ny, q.nz);
  const long long C = (long long)q.nx * q.ny * q.nz;
  const int na = q.act_x + q.act_y + q.act_z;
  const float *__restrict__ sx = q.x;
  const float *__restrict__ su = q.u;
  float *__restrict__ dx = q.y;
  float *__restrict__ du = q.thf;
  for (int r = blockIdx.x * blockDim.y + threadIdx.y; r < g.PY * g.PZ;
       r += gridDim.x * blockDim.y) {
    const int yp = r % g.PY, zp = r / g.PY;
    int y = yp - g.gy, z = zp - g.gz;
    y = y < 0 ? y + q.ny : (y >= q.ny ? y - q.ny : y);
    z = z < 0 ? z + q.nz : (z >= q.nz ? z - q.nz : z);
    const long long src = ((long long)z * q.ny + y) * q.nx;
    const long long dst = (long long)r * g.P;
    for (int xp = threadIdx.x; xp < g.P; xp += blockDim.x) {
      int x = xp - PAD_GX;
      x = x < 0 ? x + q.nx : (x >= q.nx ? x - q.nx : x);
      const float t = sx[src + x];
      float uv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < na) uv[a] = su[a * C + src + x];
      dx[dst + xp] = t;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < na) du[a * g.vol + dst + xp] = uv[a];
    }
  }
}

// Back to the box's own layout: theta (q.x) from the padded field q.y, or
// from q.thn when `alt` is set; a warp per row of the box.
__global__ void k_pad_out(const SParams<float> *__restrict__ conv, int alt) {
  const SParams<float> q = conv[blockIdx.y];
  if (q.pitch == 0) return;
  const PadGeom g = pad_geom(q.nx, q.ny, q.nz);
  const float *__restrict__ src = alt ? q.thn : q.y;
  float *__restrict__ dst = const_cast<float *>(q.x);
  for (int r = blockIdx.x * blockDim.y + threadIdx.y; r < q.ny * q.nz;
       r += gridDim.x * blockDim.y) {
    const int y = r % q.ny, z = r / q.ny;
    const long long from = ((long long)(z + g.gz) * g.PY + y + g.gy) * g.P + PAD_GX;
    const long long to = (long long)r * q.nx;
    for (int x = threadIdx.x; x < q.nx; x += blockDim.x) dst[to + x] = src[from + x];
  }
}

}  // namespace
}  // namespace fl
