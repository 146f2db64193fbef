// fl_struct_flat.cuh -- FP32 stage tile over flat runs of a plane, for the
// batched persistent kernel (fl_batch.cu).
//
// The same method and per-face arithmetic as the FP32 register tile
// (fl_struct_reg.cuh: Valle et al., Algorithm 4 with Algorithm 1's limited
// face values on Sweby's Cartesian stencil, each face flux from native_flux,
// the cell's six terms added in the TMA kernel's order x, y, z, the + face
// before the - face, so all FP32 kernels give the same bits), over a
// different unit of work: a run of consecutive cells of a plane in the flat
// order c = i + nx j, instead of a 32 x 8 rectangle.  A batch holds boxes of
// uneven sizes (32 .. 128 cells per axis): a rectangle of 32 columns wastes
// up to half of its lanes on the last column of tiles of a box, while a run
// of the flat plane only leaves the tail of the plane's last run idle.
//
//   * a warp owns CX runs of 32 cells, lane l holding cell base + l + 32 c
//     (c = 0 .. CX-1), so every load of the warp is one coalesced 128-byte
//     row of a plane;
//   * x neighbours come by warp shuffle inside a run; the two lanes at each
//     end of a run, and any cell whose neighbour wraps around the periodic x
//     end of its row, load them;
//   * the four y neighbours (flat index +- nx, +- 2 nx, periodic in y) are
//     loaded, one plane ahead with the face velocities;
//   * the z neighbours live in registers, loaded one plane ahead;
//   * a work item is (box, run of 32 CX W cells of the plane, z chunk); the
//     neighbour offsets of each cell within the plane are computed once per
//     item and reused on every plane of the chunk.
// Faces between two items are evaluated by both from the same values with
// the same code, so the update stays conservative.
#pragma once

#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_struct_reg.cuh"
#include "fl_struct_tile.cuh"

namespace fl {
namespace {

// One work item of the flat tile: run `seg` (of 32 CX blockDim.y cells) of
// every plane in z chunk `zc` of the box whose stage parameters are p.  p.
// tiles_x holds the number of runs per plane, p.zchunk the chunk length.
template <int LIM, int SEED, int CX>
__device__ __forceinline__ void stage_flat(const SParams<float> &p, int seg, int zc) {
  const int lane = threadIdx.x, w = threadIdx.y;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const unsigned plane = (unsigned)p.plane;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, nz);
  const bool need_x = p.act_x, need_y = p.act_y, need_z = p.act_z;
  const unsigned fl = (unsigned)p.flip;
  const float *__restrict__ X = p.x;
  const float *__restrict__ Ux = p.u + p.ux_off;
  const float *__restrict__ Uy = p.u + p.uy_off;
  const float *__restrict__ Uz = p.u + p.uz_off;
  const int run0 = (seg * (int)blockDim.y + w) * CX;  // first 32-cell run of the warp
  // per cell: its offset in the plane and its neighbours' (x +-1, +-2 wrap in
  // the row; y +-1, +-2 wrap in the plane)
  unsigned col[CX], xl1[CX], xl2[CX], xr1[CX], xr2[CX], ym2[CX], ym1[CX], yp1[CX], yp2[CX];
  bool valid[CX], sh_l1[CX], sh_l2[CX], sh_r1[CX], sh_r2[CX], first[CX];
#pragma unroll
  for (int c = 0; c < CX; ++c) {
    const int f = (run0 + c) * 32 + lane;
    valid[c] = f < (int)plane;
    const int g = valid[c] ? f : (int)plane - 1;
    const int y = g / nx, x = g - y * nx;
    const unsigned row = (unsigned)(y * nx);
    col[c] = (unsigned)g;
    xl1[c] = row + (unsigned)(x >= 1 ? x - 1 : x - 1 + nx);
    xl2[c] = row + (unsigned)(x >= 2 ? x - 2 : x - 2 + nx);
    xr1[c] = row + (unsigned)(x + 1 < nx ? x + 1 : x + 1 - nx);
    xr2[c] = row + (unsigned)(x + 2 < nx ? x + 2 : x + 2 - nx);
    auto ywr = [&](int d) {
      int yy = y + d;
      while (yy < 0) yy += ny;
      while (yy >= ny) yy -= ny;
      return (unsigned)(yy * nx + x);
    };
    ym2[c] = ywr(-2);
    ym1[c] = ywr(-1);
    yp1[c] = ywr(1);
    yp2[c] = ywr(2);
    // a neighbour comes by shuffle when the lane holding it is in the same
    // run and it is the cell next in the flat order (no wrap of the row), and
    // that lane's cell is inside the plane
    const int last = min(31, (int)plane - 1 - (run0 + c) * 32);  // last lane inside the plane
    sh_l1[c] = lane >= 1 && x >= 1;
    sh_l2[c] = lane >= 2 && x >= 2;
    sh_r1[c] = lane + 1 <= last && x + 1 < nx;
    sh_r2[c] = lane + 2 <= last && x + 2 < nx;
    // the -x face flux comes from the left lane's +x face unless this is the
    // run's first lane or the row's first cell (x == 0)
    first[c] = lane == 0 || x == 0;
  }
  struct Plane {
    float ym2, ym1, yp1, yp2, ux, uy, uym, uz, thn;
  };
  auto load_plane = [&](unsigned pk, Plane (&q)[CX]) {
#pragma unroll
    for (int c = 0; c < CX; ++c) {
      if (need_y) {
        q[c].ym2 = X[ym2[c] + pk];
        q[c].ym1 = X[ym1[c] + pk];
        q[c].yp1 = X[yp1[c] + pk];
        q[c].yp2 = X[yp2[c] + pk];
        q[c].uy = Uy[col[c] + pk];
        q[c].uym = Uy[ym1[c] + pk];
      }
      if (need_x) q[c].ux = Ux[col[c] + pk];
      if (need_z) q[c].uz = Uz[col[c] + pk];
      if (SEED == SEED_COMBINE) q[c].thn = p.thn[col[c] + pk];
    }
  };
  auto zw = [&](int k) -> unsigned {
    k %= nz;
    return plane * (unsigned)(k < 0 ? k + nz : k);
  };
  Plane cur[CX], nxt[CX];
  // z window per cell: planes k .. k+2, the next one prefetched, the z
  // differences and the -z face flux
  float th0[CX], thp1[CX], thp2[CX], pf[CX], dzm[CX], dz0[CX], fzp[CX];
#pragma unroll
  for (int c = 0; c < CX; ++c) {
    th0[c] = X[col[c] + plane * (unsigned)z0];
    thp1[c] = thp2[c] = pf[c] = dzm[c] = dz0[c] = fzp[c] = 0.f;
    if (need_z) {
      const float tm2 = X[col[c] + zw(z0 - 2)], tm1 = X[col[c] + zw(z0 - 1)];
      thp1[c] = X[col[c] + zw(z0 + 1)];
      thp2[c] = X[col[c] + zw(z0 + 2)];
      pf[c] = X[col[c] + zw(z0 + 3)];
      const float um = Uz[col[c] + zw(z0 - 1)];
      const float d_m2 = __fsub_rn(tm1, tm2);
      dzm[c] = __fsub_rn(th0[c], tm1);
      dz0[c] = __fsub_rn(thp1[c], th0[c]);
      fzp[c] = reg_flux<LIM>(um, tm1, th0[c], dzm[c], d_m2, dz0[c], fl);
    }
  }
  load_plane(plane * (unsigned)z0, cur);
  for (int k = z0; k < z1; ++k) {
    const unsigned pk = plane * (unsigned)k;
    if (k + 1 < z1) load_plane(pk + plane, nxt);
    const unsigned pk4 = zw(k + 4);
#pragma unroll
    for (int c = 0; c < CX; ++c) {
      float pf_next = 0.f;
      if (need_z && k + 1 < z1) pf_next = X[col[c] + pk4];
      const float t0 = th0[c];
      float acc;
      if (SEED == SEED_COMBINE) acc = __fmaf_rn(p.a, cur[c].thn, __fmul_rn(p.b, t0));
      else acc = t0;
      if (need_x) {
        const float sl1 = __shfl_up_sync(0xffffffffu, t0, 1);
        const float sl2 = __shfl_up_sync(0xffffffffu, t0, 2);
        const float sr1 = __shfl_down_sync(0xffffffffu, t0, 1);
        const float sr2 = __shfl_down_sync(0xffffffffu, t0, 2);
        const float tl1 = sh_l1[c] ? sl1 : X[xl1[c] + pk];
        const float tl2 = sh_l2[c] ? sl2 : X[xl2[c] + pk];
        const float tr1 = sh_r1[c] ? sr1 : X[xr1[c] + pk];
        const float tr2 = sh_r2[c] ? sr2 : X[xr2[c] + pk];
        const float dm1 = __fsub_rn(t0, tl1), d0 = __fsub_rn(tr1, t0);
        const float dp1 = __fsub_rn(tr2, tr1), dm2 = __fsub_rn(tl1, tl2);
        const float fp = reg_flux<LIM>(cur[c].ux, t0, tr1, d0, dm1, dp1, fl);
        float fm = __shfl_up_sync(0xffffffffu, fp, 1);
        if (first[c]) fm = reg_flux<LIM>(Ux[xl1[c] + pk], tl1, t0, dm1, dm2, d0, fl);
        acc = __fmaf_rn(-p.cx, fp, acc);
        acc = __fmaf_rn(p.cx, fm, acc);
      }
      if (need_y) {
        const Plane &q = cur[c];
        const float dm2 = __fsub_rn(q.ym1, q.ym2), dm1 = __fsub_rn(t0, q.ym1);
        const float d0 = __fsub_rn(q.yp1, t0), dp1 = __fsub_rn(q.yp2, q.yp1);
        const float fm = reg_flux<LIM>(q.uym, q.ym1, t0, dm1, dm2, d0, fl);
        const float fp = reg_flux<LIM>(q.uy, t0, q.yp1, d0, dm1, dp1, fl);
        acc = __fmaf_rn(-p.cy, fp, acc);
        acc = __fmaf_rn(p.cy, fm, acc);
      }
      float dzp = 0.f, fz = 0.f;
      if (need_z) {
        dzp = __fsub_rn(thp2[c], thp1[c]);
        fz = reg_flux<LIM>(cur[c].uz, t0, thp1[c], dz0[c], dzm[c], dzp, fl);
        acc = __fmaf_rn(-p.cz, fz, acc);
        acc = __fmaf_rn(p.cz, fzp[c], acc);
      }
      if (valid[c]) p.y[col[c] + pk] = acc;
      if (need_z) {
        fzp[c] = fz;
        dzm[c] = dz0[c];
        dz0[c] = dzp;
        th0[c] = thp1[c];
        thp1[c] = thp2[c];
        thp2[c] = pf[c];
        pf[c] = pf_next;
      } else if (k + 1 < z1) {
        th0[c] = X[col[c] + pk + plane];
      }
    }
#pragma unroll
    for (int c = 0; c < CX; ++c) cur[c] = nxt[c];
  }
}

}  // namespace
}  // namespace fl
