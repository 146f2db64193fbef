// fl_struct_tma.cu -- FP32 fused limited-convection stage with TMA-staged
// planes, for periodic Cartesian meshes with nx % 4 == 0, nx >= 128 and
// ny >= 8; other shapes use the kernel of fl_structured.cu.
//
// Same method as fl_structured.cu (Valle et al., Algorithm 4 with the
// limited face values of Algorithm 1, Sweby's stencil on Cartesian grids).
// FP32 is bandwidth-bound on this part, so the kernel is built to spend few
// instructions per cell and keep several planes of loads in flight:
//   * a CTA owns a 128 x 8 column of cells and streams through z; a consumer
//     thread owns four consecutive x cells of one row (128-bit loads and
//     stores);
//   * a ninth warp is the producer: one lane issues, per plane, the TMA tile
//     copies (cp.async.bulk.tensor) of the theta tile and its periodic halos
//     (4-wide x boxes, one-row y boxes at wrapped coordinates), the u_f
//     tiles with their -x / -y halo faces and theta^n, completing on the
//     slot's "full" mbarrier; a ring of 3 slots keeps two planes in flight;
//   * consumer warps never wait for one another: each waits on the slot's
//     full barrier, computes, and arrives on the slot's "empty" barrier,
//     which the producer waits on before refilling the slot;
//   * x neighbours move between lanes by warp shuffles (only the warp-edge
//     lanes read the halo boxes); each x face is evaluated once, the -x
//     face of a lane's first cell arriving by shuffle from the lane to its
//     left (lane 0 evaluates its own);
//   * each thread evaluates both y faces of its cells (the +y face of one
//     row is the -y face of the next, computed by another warp from the same
//     values with the same code, so both sides see bit-identical fluxes) and
//     the +z face; the -z face is the previous plane's, kept in a register;
//   * the limiter runs on FP32 min/max (native_flux).
// Every mbarrier wait is bounded: on expiry the warp records FL_ETIMEOUT in
// the mesh status word and stops; the producer stops issuing and waits
// (bounded again) for the copies it has in flight before it returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"

namespace fl {

namespace {

constexpr int TX = 128, VX = 4, LANES = TX / VX, TY = 8;
#ifndef FL_TMA_RING
#define FL_TMA_RING 4
#endif
#ifndef FL_TMA_MINB
#define FL_TMA_MINB 2
#endif
#ifndef FL_TMA_UNROLL
#define FL_TMA_UNROLL 1
#endif
constexpr int RING = FL_TMA_RING, MINB = FL_TMA_MINB, UNROLL = FL_TMA_UNROLL;
// slot layout (bytes); every TMA destination is 128-byte aligned
constexpr int OFF_TH = 0;       // [8][128] theta
constexpr int OFF_XL = 4096;    // [8][4]   theta x0-4 .. x0-1
constexpr int OFF_XR = 4224;    // [8][4]   theta x0+w .. x0+w+3
constexpr int OFF_YT = 4352;    // [2][128] theta rows y0-2, y0-1
constexpr int OFF_YB = 5376;    // [2][128] theta rows y0+h, y0+h+1 (one box each)
constexpr int OFF_UX = 6400;    // [8][128] u of +x faces
constexpr int OFF_UXH = 10496;  // [8][4]   u of x faces x0-4 .. x0-1
constexpr int OFF_UY = 10624;   // [8][128] u of +y faces
constexpr int OFF_UYH = 14720;  // [1][128] u of y faces of row y0-1
constexpr int OFF_UZ = 15232;   // [8][128] u of +z faces
constexpr int OFF_THN = 19328;  // [8][128] theta^n
constexpr int SLOT = 23424;
constexpr long long WAIT_LIMIT = 1LL << 22;  // try_wait polls before giving up

struct TParams {
  const float *x;  // plain loads of the z neighbours
  const float *u;
  float *y;
  int nx, ny, nz;
  int act_z;
  int bx_u, by_u, bz_u;  // u_f block of each axis
  long long uz_off;
  float cx, cy, cz, a, b;
  int tiles_x, tiles_y, zchunk;
  int *status;
  int zlo, zhi;  // the tiles cover planes [zlo, zhi)
  int ylo, yhi;  // and rows [ylo, yhi) of them
};

__device__ __forceinline__ uint32_t sa(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sa(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                     int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sa(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
      : "memory");
}

__device__ __forceinline__ void tma4(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                     int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(sa(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(sa(bar))
      : "memory");
}

__device__ __forceinline__ int wrapv(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// flux of a face from its Delta a, the two candidate upstream Deltas and
// the two candidate upwind values (picked by the sign of u: u > 0 is false
// for 0, -0 and NaN, the selection rule of the scalar path)
template <int LIM>
__device__ __forceinline__ float flux(float u, float thC_pos, float thC_neg, float a, float b_pos,
                                      float b_neg) {
  const bool sp = u > 0.0f;
  return native_flux<LIM>(u, sp ? thC_pos : thC_neg, a, sp ? b_pos : b_neg);
}

__device__ __forceinline__ float4 ld4(const unsigned char *base, int off_bytes) {
  return *reinterpret_cast<const float4 *>(base + off_bytes);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}

// k mod n for k in [0, 2n) without a division (n >= 4 here in practice)
__device__ __forceinline__ int wrap_up(int k, int n) {
  if (k >= n) k -= n;
  return k < n ? k : k % n;
}

template <int LIM, int SEED>
__global__ void __launch_bounds__(LANES *(TY + 1), MINB) k_struct_stage_tma(
    const TParams p, const __grid_constant__ CUtensorMap m_th,
    const __grid_constant__ CUtensorMap m_thx, const __grid_constant__ CUtensorMap m_thy2,
    const __grid_constant__ CUtensorMap m_thy1, const __grid_constant__ CUtensorMap m_u,
    const __grid_constant__ CUtensorMap m_ux, const __grid_constant__ CUtensorMap m_uy1,
    const __grid_constant__ CUtensorMap m_thn) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[RING];
  __shared__ __align__(8) uint64_t empty[RING];
  const int lane = threadIdx.x, ty = threadIdx.y;
  int bid = blockIdx.x;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = p.ylo + by * TY;
  const int z0 = p.zlo + bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.zhi);
  const int L = z1 - z0;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int w = min(TX, nx - x0), h = min(TY, p.yhi - y0);  // w is a multiple of 4
  const bool az = p.act_z;
  auto parity = [](int q) { return (uint32_t)((q / RING) & 1); };

  if (lane == 0 && ty == 0) {
    for (int i = 0; i < RING; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], TY);  // one arrival per consumer warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // ================================================================ producer
  if (ty == TY) {
    if (lane != 0) return;
    // wrapped halo coordinates, fixed for the CTA
    const int cxl = wrapv(x0 - 4, nx), cxr = wrapv(x0 + w, nx);
    const int cyt = wrapv(y0 - 2, ny), cyh = wrapv(y0 - 1, ny);
    const int cyb0 = wrapv(y0 + h, ny), cyb1 = wrapv(y0 + h + 1, ny);
    uint32_t bytes = 4096 + 256 + 1024 + 1024 + 4096 + 128 + 4096 + 512;
    if (az) bytes += 4096;
    if (SEED == 1) bytes += 4096;
    int issued = 0;
    for (int q = 0; q < L; ++q) {
      const int slot = q % RING;
      if (q >= RING && !mbar_wait(&empty[slot], parity(q - RING))) {
        record_status(p.status, (int)FL_ETIMEOUT);
        break;
      }
      unsigned char *s = smem + slot * SLOT;
      uint64_t *bar = &full[slot];
      const int pz = z0 + q;
      // the slot was last read through the generic proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect(bar, bytes);
      tma3(s + OFF_TH, &m_th, bar, x0, y0, pz);
      tma3(s + OFF_XL, &m_thx, bar, cxl, y0, pz);
      tma3(s + OFF_XR, &m_thx, bar, cxr, y0, pz);
      tma3(s + OFF_YT, &m_thy2, bar, x0, cyt, pz);
      // the two rows below may straddle the periodic end: one box each
      tma3(s + OFF_YB, &m_thy1, bar, x0, cyb0, pz);
      tma3(s + OFF_YB + 512, &m_thy1, bar, x0, cyb1, pz);
      tma4(s + OFF_UX, &m_u, bar, x0, y0, pz, p.bx_u);
      tma4(s + OFF_UXH, &m_ux, bar, cxl, y0, pz, p.bx_u);
      tma4(s + OFF_UY, &m_u, bar, x0, y0, pz, p.by_u);
      tma4(s + OFF_UYH, &m_uy1, bar, x0, cyh, pz, p.by_u);
      if (az) tma4(s + OFF_UZ, &m_u, bar, x0, y0, pz, p.bz_u);
      if (SEED == 1) tma3(s + OFF_THN, &m_thn, bar, x0, y0, pz);
      issued = q + 1;
    }
    // before the CTA may end: the last copy issued into each slot has landed
    for (int q = max(0, issued - RING); q < issued; ++q)
      if (!mbar_wait(&full[q % RING], parity(q))) record_status(p.status, (int)FL_ETIMEOUT);
    return;
  }

  // =============================================================== consumers
  const int last_lane = w / VX - 1;
  const bool valid = lane <= last_lane && ty < h;
  // z window of the thread's four cells by plain 128-bit loads
  // 32-bit element offsets from the field base pointers (below n_cells < 2^31)
  const unsigned plane = (unsigned)nx * (unsigned)ny;
  const int cxv = min(x0 + VX * lane, nx - VX), cyv = min(y0 + ty, ny - 1);
  const unsigned col = (unsigned)cxv + (unsigned)nx * (unsigned)cyv;
  auto X4 = [&](int k) {  // k in [0, nz)
    return *reinterpret_cast<const float4 *>(p.x + (col + plane * (unsigned)k));
  };
  float th0[4], thp1[4] = {0, 0, 0, 0}, thp2[4] = {0, 0, 0, 0}, dzm[4] = {0, 0, 0, 0},
        dz0[4] = {0, 0, 0, 0}, fzp[4] = {0, 0, 0, 0};
  float4 pf = make_float4(0, 0, 0, 0);
  {
    const float4 c0 = X4(z0);
    th0[0] = c0.x;
    th0[1] = c0.y;
    th0[2] = c0.z;
    th0[3] = c0.w;
  }
  if (az) {
    const float4 m2 = X4(wrapv(z0 - 2, nz)), m1 = X4(wrapv(z0 - 1, nz));
    const float4 p1 = X4(wrapv(z0 + 1, nz)), p2 = X4(wrapv(z0 + 2, nz));
    pf = X4(wrapv(z0 + 3, nz));
    const float4 um = *reinterpret_cast<const float4 *>(
        p.u + p.uz_off + (col + plane * (unsigned)wrapv(z0 - 1, nz)));
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
      fzp[v] = flux<LIM>(uzm[v], tm1[v], th0[v], dzm[v], d_m2, dz0[v]);
    }
  }

  const int rowb = ty * TX * 4 + lane * VX * 4;  // byte offset of the thread's cells in a row tile
  // y rows ty-2 .. ty+2 of the slot (fixed per thread)
  int yoff[5];
#pragma unroll
  for (int dd = -2; dd <= 2; ++dd) {
    const int r = ty + dd;
    int off;
    if (r < 0) off = OFF_YT + (2 + r) * TX * 4;
    else if (r < h) off = OFF_TH + r * TX * 4;
    else off = OFF_YB + min(r - h, 1) * TX * 4;
    yoff[dd + 2] = off + lane * VX * 4;
  }
  const int umoff = (ty > 0) ? OFF_UY + rowb - TX * 4 : OFF_UYH + lane * VX * 4;
  int knext = wrap_up(z0 + 4, nz);  // plane of the next z-window load
  // unrolled so that the z-window shifts become register renaming
#pragma unroll UNROLL
  for (int q = 0; q < L; ++q) {
    const int k = z0 + q;
    const int slot = q % RING;
    float4 pf_next = make_float4(0, 0, 0, 0);
    if (az && q + 1 < L) {
      pf_next = X4(knext);
      knext = (knext + 1 == nz) ? 0 : knext + 1;
    }
    {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[slot], parity(q)));
      if (!ok) {
        if (lane == 0) record_status(p.status, (int)FL_ETIMEOUT);
        return;
      }
    }
    const unsigned char *s = smem + slot * SLOT;
    float acc[4];
    if (SEED == 1) {
      const float4 tn = ld4(s, OFF_THN + rowb);
      const float tnv[4] = {tn.x, tn.y, tn.z, tn.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = __fmaf_rn(p.a, tnv[v], __fmul_rn(p.b, th0[v]));
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = th0[v];
    }
    // ------------------------------------------------------ x faces
    {
      const float4 c = ld4(s, OFF_TH + rowb);
      float t[8];  // theta at offsets -2 .. 5 from the first cell
      t[2] = c.x;
      t[3] = c.y;
      t[4] = c.z;
      t[5] = c.w;
      const float l2 = __shfl_up_sync(0xffffffffu, c.z, 1);
      const float l1 = __shfl_up_sync(0xffffffffu, c.w, 1);
      const float r0 = __shfl_down_sync(0xffffffffu, c.x, 1);
      const float r1 = __shfl_down_sync(0xffffffffu, c.y, 1);
      const float *xl = reinterpret_cast<const float *>(s + OFF_XL) + ty * 4;
      const float *xr = reinterpret_cast<const float *>(s + OFF_XR) + ty * 4;
      t[0] = (lane == 0) ? xl[2] : l2;
      t[1] = (lane == 0) ? xl[3] : l1;
      t[6] = (lane == last_lane) ? xr[0] : r0;
      t[7] = (lane == last_lane) ? xr[1] : r1;
      float d[7];  // d[m + 2] = Delta of face m (between offsets m and m + 1)
#pragma unroll
      for (int m = -2; m <= 4; ++m) d[m + 2] = __fsub_rn(t[m + 3], t[m + 2]);
      const float4 ux = ld4(s, OFF_UX + rowb);
      const float uv[4] = {ux.x, ux.y, ux.z, ux.w};
      float fx[5];  // fx[m + 1] = flux of face m, m = -1 .. 3
#pragma unroll
      for (int m = 0; m < 4; ++m)
        fx[m + 1] = flux<LIM>(uv[m], t[m + 2], t[m + 3], d[m + 2], d[m + 1], d[m + 3]);
      fx[0] = __shfl_up_sync(0xffffffffu, fx[4], 1);
      if (lane == 0) {
        const float um = reinterpret_cast<const float *>(s + OFF_UXH)[ty * 4 + 3];
        fx[0] = flux<LIM>(um, t[1], t[2], d[1], d[0], d[2]);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        acc[v] = __fmaf_rn(-p.cx, fx[v + 1], acc[v]);
        acc[v] = __fmaf_rn(p.cx, fx[v], acc[v]);
      }
    }
    // ------------------------------------------------------ y faces
    {
      float4 r4[5];  // rows ty-2 .. ty+2 at the thread's four columns
#pragma unroll
      for (int dd = 0; dd < 5; ++dd) r4[dd] = ld4(s, yoff[dd]);
      const float4 up4 = ld4(s, OFF_UY + rowb);
      const float4 um4 = ld4(s, umoff);
      const float upv[4] = {up4.x, up4.y, up4.z, up4.w}, umv[4] = {um4.x, um4.y, um4.z, um4.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float yv[5] = {(&r4[0].x)[v], (&r4[1].x)[v], (&r4[2].x)[v], (&r4[3].x)[v],
                             (&r4[4].x)[v]};
        const float dm2 = __fsub_rn(yv[1], yv[0]), dm1 = __fsub_rn(yv[2], yv[1]);
        const float d0 = __fsub_rn(yv[3], yv[2]), dp1 = __fsub_rn(yv[4], yv[3]);
        const float fm = flux<LIM>(umv[v], yv[1], yv[2], dm1, dm2, d0);
        const float fp = flux<LIM>(upv[v], yv[2], yv[3], d0, dm1, dp1);
        acc[v] = __fmaf_rn(-p.cy, fp, acc[v]);
        acc[v] = __fmaf_rn(p.cy, fm, acc[v]);
      }
    }
    // ------------------------------------------------------ z face
    float dzp[4] = {0, 0, 0, 0}, fz[4] = {0, 0, 0, 0};
    if (az) {
      const float4 uz4 = ld4(s, OFF_UZ + rowb);
      const float uzv[4] = {uz4.x, uz4.y, uz4.z, uz4.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        dzp[v] = __fsub_rn(thp2[v], thp1[v]);
        fz[v] = flux<LIM>(uzv[v], th0[v], thp1[v], dz0[v], dzm[v], dzp[v]);
        acc[v] = __fmaf_rn(-p.cz, fz[v], acc[v]);
        acc[v] = __fmaf_rn(p.cz, fzp[v], acc[v]);
      }
    }
    // this warp is done with the slot
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
    if (valid)
      *reinterpret_cast<float4 *>(p.y + (col + plane * (unsigned)k)) =
          make_float4(acc[0], acc[1], acc[2], acc[3]);
    // ------------------------------------------------------ rotate z
    if (az) {
      const float pv[4] = {pf.x, pf.y, pf.z, pf.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fzp[v] = fz[v];
        dzm[v] = dz0[v];
        dz0[v] = dzp[v];
        th0[v] = thp1[v];
        thp1[v] = thp2[v];
        thp2[v] = pv[v];
      }
      pf = pf_next;
    } else if (q + 1 < L) {
      const float4 c0 = X4(k + 1);
      th0[0] = c0.x;
      th0[1] = c0.y;
      th0[2] = c0.z;
      th0[3] = c0.w;
    }
  }
}

// --------------------------------------------------------------- host side
typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn get_encode() {
  static encode_fn fn = []() -> encode_fn {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<encode_fn>(f);
  }();
  return fn;
}

bool encode(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box) {
  encode_fn fn = get_encode();
  if (!fn) return false;
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int LIM, int SEED>
cudaError_t launch(const TParams &p, const CUtensorMap *maps, unsigned grid, cudaStream_t st) {
  auto k = k_struct_stage_tma<LIM, SEED>;
  const int smem = RING * SLOT;
  const cudaError_t e = set_smem_limit(reinterpret_cast<const void *>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<grid, dim3(LANES, TY + 1), smem, st>>>(p, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5],
                                         maps[6], maps[7]);
  return cudaGetLastError();
}

template <int SEED>
cudaError_t launch_lim(int lim, const TParams &p, const CUtensorMap *maps, unsigned grid,
                       cudaStream_t st) {
  switch (lim) {
    case LIM_UPWIND: return launch<LIM_UPWIND, SEED>(p, maps, grid, st);
    case LIM_CENTRAL: return launch<LIM_CENTRAL, SEED>(p, maps, grid, st);
    case LIM_MINMOD: return launch<LIM_MINMOD, SEED>(p, maps, grid, st);
    case LIM_VANLEER: return launch<LIM_VANLEER, SEED>(p, maps, grid, st);
    case LIM_SUPERBEE: return launch<LIM_SUPERBEE, SEED>(p, maps, grid, st);
    case LIM_SMART: return launch<LIM_SMART, SEED>(p, maps, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool struct_tma_eligible(const fl_mesh *m, const StageArgs &s) {
  // a negative velocity factor (reversed flow) needs the flipped upwind
  // test of the plain kernel
  if (m->kind != 0 || s.seed == 2 || !(s.g >= 0)) return false;
  if (m->nx % 4 != 0 || m->nx < TX || m->ny < TY) return false;
  if (!m->status) return false;
  const uintptr_t mask = 15;
  if (((uintptr_t)s.x & mask) || ((uintptr_t)s.u & mask) || ((uintptr_t)s.y & mask)) return false;
  if (s.seed == 1 && ((uintptr_t)s.thn & mask)) return false;
  return get_encode() != nullptr;
}

cudaError_t struct_stage_tma(const fl_mesh *m, int lim, const StageArgs &s, cudaStream_t st) {
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  const cuuint64_t plane = (cuuint64_t)nx * ny;
  const int nblk = m->act[0] + m->act[1] + m->act[2];
  const cuuint64_t d3[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t s3[2] = {(cuuint64_t)nx * 4, plane * 4};
  const cuuint64_t d4[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)nblk};
  const cuuint64_t s4[3] = {(cuuint64_t)nx * 4, plane * 4, plane * nz * 4};
  const cuuint32_t bmain[4] = {TX, TY, 1, 1}, bx[4] = {4, TY, 1, 1}, by2[4] = {TX, 2, 1, 1},
                   by1[4] = {TX, 1, 1, 1};
  alignas(64) CUtensorMap maps[8];
  bool ok = encode(&maps[0], s.x, 3, d3, s3, bmain) && encode(&maps[1], s.x, 3, d3, s3, bx) &&
            encode(&maps[2], s.x, 3, d3, s3, by2) && encode(&maps[3], s.x, 3, d3, s3, by1) &&
            encode(&maps[4], s.u, 4, d4, s4, bmain) && encode(&maps[5], s.u, 4, d4, s4, bx) &&
            encode(&maps[6], s.u, 4, d4, s4, by1) &&
            encode(&maps[7], s.seed == 1 ? s.thn : s.x, 3, d3, s3, bmain);
  if (!ok) return cudaErrorNotSupported;  // caller falls back to the plain kernel
  TParams p;
  p.x = static_cast<const float *>(s.x);
  p.u = static_cast<const float *>(s.u);
  p.y = static_cast<float *>(s.y);
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.act_z = m->act[2];
  p.bx_u = (int)(m->u_off[0] / m->C);
  p.by_u = (int)(m->u_off[1] / m->C);
  p.bz_u = (int)(m->u_off[2] / m->C);
  p.uz_off = m->u_off[2];
  const double sc = ((s.seed == 0) ? s.dt : s.b * s.dt) * s.g;
  p.cx = (float)(sc / m->hx);
  p.cy = (float)(sc / m->hy);
  p.cz = (float)(sc / m->hz);
  p.a = blend_a<float>(s.a, s.b);
  p.b = (float)s.b;
  p.tiles_x = (nx + TX - 1) / TX;
  p.ylo = s.yhi < 0 ? 0 : s.ylo;
  p.yhi = s.yhi < 0 ? ny : s.yhi;
  p.tiles_y = (p.yhi - p.ylo + TY - 1) / TY;
  const long long cols = (long long)p.tiles_x * p.tiles_y;
  // whole waves of co-resident CTAs (the occupancy query needs the kernel's
  // dynamic shared-memory limit raised first)
  if (set_smem_limit(reinterpret_cast<const void *>(&k_struct_stage_tma<LIM_SUPERBEE, 1>),
                     RING * SLOT) != cudaSuccess)
    return cudaErrorNotSupported;
  const int resident = resident_ctas(reinterpret_cast<const void *>(&k_struct_stage_tma<LIM_SUPERBEE, 1>),
                                     LANES * (TY + 1), RING * SLOT);
  p.zlo = s.zhi < 0 ? 0 : s.zlo;
  p.zhi = s.zhi < 0 ? nz : s.zhi;
  const int nzr = p.zhi - p.zlo;
  const int zchunk = pick_zchunk(cols, nzr, resident, 3);
  p.zchunk = zchunk;
  p.status = m->status;
  const unsigned grid = (unsigned)(cols * ((nzr + zchunk - 1) / zchunk));
  return s.seed == 0 ? launch_lim<0>(lim, p, maps, grid, st) : launch_lim<1>(lim, p, maps, grid, st);
}

}  // namespace fl
