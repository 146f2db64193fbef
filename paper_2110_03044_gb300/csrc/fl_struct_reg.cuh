// fl_struct_reg.cuh -- FP32 tile of the fused limited-convection stage with
// no shared memory and no barriers (periodic Cartesian meshes of any size).
//
// Same method and the same 32 x 8 tiles as fl_struct_tile.cuh (Valle et
// al., Algorithm 4 with the limited face values of Algorithm 1 on Sweby's
// Cartesian stencil), for FP32, where the shared-memory tile's three
// barriers per plane leave the stage latency-bound:
//   * a warp owns one row of 32 cells of the tile; a thread owns one cell
//     and streams through the tile's z chunk;
//   * x neighbours come from warp shuffles; the warp-edge lanes (and lanes
//     whose neighbour lies past a ragged end of the mesh) load theirs;
//   * the four y neighbours are loaded directly (the rows are shared with
//     the neighbouring warps through L1), one plane ahead with the face
//     velocities;
//   * the z neighbours live in registers, loaded one plane ahead;
//   * each face flux uses FP32 min/max (native_flux) and the
//     accumulation order of the TMA kernel (fl_struct_tma.cu: x, y, z; the
//     + face before the - face), so both kernels give the same bits.
// Each x face is evaluated once per warp (the -x face of a cell arrives by
// shuffle; lane 0 evaluates its own); both y faces and the +z face are
// evaluated per cell.  Faces on a tile edge are computed by both tiles from
// the same values with the same code, so the update stays conservative.
#pragma once

#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_struct_tile.cuh"

namespace fl {
namespace {

// flux of a face from its Delta a, the two candidate upstream Deltas and the
// two candidate upwind values (picked by the sign of u: u > 0 is false for
// 0, -0 and NaN)
// (flip: sign mask of a negative velocity factor, toggled into u for the test)
template <int LIM>
__device__ __forceinline__ float reg_flux(float u, float thC_pos, float thC_neg, float a,
                                          float b_pos, float b_neg, unsigned flip) {
  const bool sp = __uint_as_float(__float_as_uint(u) ^ flip) > 0.0f;
  return native_flux<LIM>(u, sp ? thC_pos : thC_neg, a, sp ? b_pos : b_neg, flip);
}

// reg_flux with van Leer's quotient unchecked (FT<float>::quot_unchecked):
// the same value wherever `far` stays clear
template <int LIM>
__device__ __forceinline__ float reg_flux_unchecked(float u, float thC_pos, float thC_neg, float a,
                                                    float b_pos, float b_neg, unsigned flip,
                                                    bool &far) {
  const bool sp = __uint_as_float(__float_as_uint(u) ^ flip) > 0.0f;
  return native_flux_q<LIM>(u, sp ? thC_pos : thC_neg, a, sp ? b_pos : b_neg, flip,
                            [&far](float n, float s, bool need) {
                              return FT<float>::quot_unchecked(n, s, need, far);
                            });
}

template <int LIM, int SEED>
__device__ __forceinline__ void stage_tile_reg(const SParams<float> &p, int tile) {
  const int lane = threadIdx.x, ty = threadIdx.y;
  int bid = tile;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = p.ylo + by * (int)blockDim.y;
  const int z0 = p.zlo + bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, min(p.nz, p.zhi));
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int last = min(TX, nx - x0) - 1;  // last lane inside the mesh
  const bool valid = lane <= last && y0 + ty < min(ny, p.yhi);
  const int x = x0 + min(lane, last);
  const int y = min(y0 + ty, ny - 1);
  const bool need_x = p.act_x, need_y = p.act_y, need_z = p.act_z;
  // Addressing: one 64-bit base pointer per stream, computed once, plus
  // 32-bit element offsets (a plane offset plane * k is below n_cells <
  // 2^31), so that each load costs one wide multiply-add instead of 64-bit
  // index arithmetic (which had been about 40 % of the tile's instructions)
  const unsigned plane = (unsigned)p.plane;
  auto wr = [](int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
  };
  const unsigned rowy = (unsigned)nx * (unsigned)y;
  const unsigned col = (unsigned)x + rowy;
  const int xl1 = wr(x - 1, nx), xl2 = wr(x - 2, nx), xr1 = wr(x + 1, nx), xr2 = wr(x + 2, nx);
  const unsigned ym2 = (unsigned)nx * wr(y - 2, ny) + x, ym1 = (unsigned)nx * wr(y - 1, ny) + x;
  const unsigned yp1 = (unsigned)nx * wr(y + 1, ny) + x, yp2 = (unsigned)nx * wr(y + 2, ny) + x;
  // which x neighbours come by shuffle (the lane holding them is inside)
  const bool sh_l1 = lane >= 1, sh_l2 = lane >= 2;
  const bool sh_r1 = lane + 1 <= last, sh_r2 = lane + 2 <= last;
  const float *__restrict__ X = p.x;
  const float *__restrict__ Ux = p.u + p.ux_off;
  const float *__restrict__ Uy = p.u + p.uy_off;
  const float *__restrict__ Uz = p.u + p.uz_off;
  const unsigned fl = (unsigned)p.flip;
  // the plane's loads, issued one plane ahead
  struct Plane {
    float ym2, ym1, yp1, yp2, ux, uy, uym, uz, thn;
  };
  auto load_plane = [&](unsigned pk, Plane &q) {
    if (need_y) {
      q.ym2 = X[ym2 + pk];
      q.ym1 = X[ym1 + pk];
      q.yp1 = X[yp1 + pk];
      q.yp2 = X[yp2 + pk];
      q.uy = Uy[col + pk];
      q.uym = Uy[ym1 + pk];
    }
    if (need_x) q.ux = Ux[col + pk];
    if (need_z) q.uz = Uz[col + pk];
    if (SEED == SEED_COMBINE) q.thn = p.thn[col + pk];
  };
  Plane cur{}, nxt{};

  // ---- z window at (x, y): planes k-1 .. k+2, the next one prefetched
  float th0, thp1 = 0.f, thp2 = 0.f, pf = 0.f, dzm = 0.f, dz0 = 0.f, fzp = 0.f;
  th0 = X[col + plane * z0];
  if (need_z) {
    const float tm2 = X[col + plane * wr(z0 - 2, nz)], tm1 = X[col + plane * wr(z0 - 1, nz)];
    thp1 = X[col + plane * wr(z0 + 1, nz)];
    thp2 = X[col + plane * wr(z0 + 2, nz)];
    pf = X[col + plane * wr(z0 + 3, nz)];
    const float um = Uz[col + plane * wr(z0 - 1, nz)];
    const float d_m2 = __fsub_rn(tm1, tm2);
    dzm = __fsub_rn(th0, tm1);
    dz0 = __fsub_rn(thp1, th0);
    fzp = reg_flux<LIM>(um, tm1, th0, dzm, d_m2, dz0, fl);
  }
  load_plane(plane * z0, cur);
  for (int k = z0; k < z1; ++k) {
    const unsigned pk = plane * k;
    if (k + 1 < z1) load_plane(pk + plane, nxt);
    float pf_next = 0.f;
    if (need_z && k + 1 < z1) {
      int kn = k + 4;  // k + 4 < 2 nz unless nz < 4
      if (kn >= nz) kn -= nz;
      if (kn >= nz) kn %= nz;
      pf_next = X[col + plane * kn];
    }
    float acc;
    if (SEED == SEED_COMBINE) acc = __fmaf_rn(p.a, cur.thn, __fmul_rn(p.b, th0));
    else acc = th0;
    // ------------------------------------------------------ x faces
    if (need_x) {
      const float sl1 = __shfl_up_sync(0xffffffffu, th0, 1);
      const float sl2 = __shfl_up_sync(0xffffffffu, th0, 2);
      const float sr1 = __shfl_down_sync(0xffffffffu, th0, 1);
      const float sr2 = __shfl_down_sync(0xffffffffu, th0, 2);
      const float tl1 = sh_l1 ? sl1 : X[rowy + xl1 + pk];
      const float tl2 = sh_l2 ? sl2 : X[rowy + xl2 + pk];
      const float tr1 = sh_r1 ? sr1 : X[rowy + xr1 + pk];
      const float tr2 = sh_r2 ? sr2 : X[rowy + xr2 + pk];
      const float dm1 = __fsub_rn(th0, tl1), d0 = __fsub_rn(tr1, th0);
      const float dp1 = __fsub_rn(tr2, tr1), dm2 = __fsub_rn(tl1, tl2);
      // +x face of the cell (between x and x+1)
      const float fp = reg_flux<LIM>(cur.ux, th0, tr1, d0, dm1, dp1, fl);
      // -x face: the left lane's +x face, lane 0 its own
      float fm = __shfl_up_sync(0xffffffffu, fp, 1);
      if (lane == 0)
        fm = reg_flux<LIM>(Ux[rowy + xl1 + pk], tl1, th0, dm1, dm2, d0, fl);
      acc = __fmaf_rn(-p.cx, fp, acc);
      acc = __fmaf_rn(p.cx, fm, acc);
    }
    // ------------------------------------------------------ y faces
    if (need_y) {
      const float dm2 = __fsub_rn(cur.ym1, cur.ym2), dm1 = __fsub_rn(th0, cur.ym1);
      const float d0 = __fsub_rn(cur.yp1, th0), dp1 = __fsub_rn(cur.yp2, cur.yp1);
      const float fm = reg_flux<LIM>(cur.uym, cur.ym1, th0, dm1, dm2, d0, fl);
      const float fp = reg_flux<LIM>(cur.uy, th0, cur.yp1, d0, dm1, dp1, fl);
      acc = __fmaf_rn(-p.cy, fp, acc);
      acc = __fmaf_rn(p.cy, fm, acc);
    }
    // ------------------------------------------------------ z face
    float dzp = 0.f, fz = 0.f;
    if (need_z) {
      dzp = __fsub_rn(thp2, thp1);
      fz = reg_flux<LIM>(cur.uz, th0, thp1, dz0, dzm, dzp, fl);
      acc = __fmaf_rn(-p.cz, fz, acc);
      acc = __fmaf_rn(p.cz, fzp, acc);
    }
    if (valid) p.y[col + pk] = acc;
    cur = nxt;
    // ------------------------------------------------------ rotate z
    if (need_z) {
      fzp = fz;
      dzm = dz0;
      dz0 = dzp;
      th0 = thp1;
      thp1 = thp2;
      thp2 = pf;
      pf = pf_next;
    } else if (k + 1 < z1) {
      th0 = X[col + plane * (k + 1)];
    }
  }
}

}  // namespace
}  // namespace fl
