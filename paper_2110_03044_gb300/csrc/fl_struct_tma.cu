// fl_struct_tma.cu -- FP32 fused limited-convection stage with TMA-staged
// planes, for periodic Cartesian meshes with nx % 4 == 0, nx >= 32 and (when
// y is active) ny >= 8; other shapes use the kernel of fl_structured.cu.
//
// Same method as fl_structured.cu (Valle et al., Algorithm 4 with the
// limited face values of Algorithm 1, Sweby's stencil on Cartesian grids);
// this variant is built for the bandwidth-bound FP32 case:
//   * one thread per cell of a 32 x 8 column, streaming through z;
//   * for every plane, one elected thread issues the TMA tile copies
//     (cp.async.bulk.tensor) of the plane's theta tile and its periodic halos
//     (4-wide x boxes and 2-row y boxes at wrapped coordinates), the three
//     u_f tiles with their -x / -y halo faces and theta^n, all completing on
//     the slot's mbarrier; a ring of 4 slots keeps three planes in flight
//     beyond the one being computed;
//   * the z neighbours of a column come from plain loads two planes ahead;
//   * each thread evaluates both x faces and both y faces of its cell
//     (recomputing a neighbour's face costs a few FP32 operations and saves
//     the shared-memory exchange and its barriers); the z face below comes
//     from the previous plane in a register.  The two threads that evaluate
//     a face do so with the same code on the same values, so the flux is
//     bit-identical on both sides and the update conserves;
//   * one barrier per plane, before the slot is refilled.
// Every mbarrier wait is bounded: on expiry the CTA records FL_ETIMEOUT in
// the mesh status word, waits (bounded again) for its copies in flight and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"

namespace fl {

namespace {

constexpr int TX = 32, TY = 8, RING = 4;
// slot layout (bytes); every TMA destination is 128-byte aligned
constexpr int OFF_TH = 0;      // [8][32] theta
constexpr int OFF_XL = 1024;   // [8][4]  theta x0-4 .. x0-1
constexpr int OFF_XR = 1152;   // [8][4]  theta x0+w .. x0+w+3
constexpr int OFF_YT = 1280;   // [2][32] theta rows y0-2, y0-1
constexpr int OFF_YB = 1536;   // [2][32] theta rows y0+h, y0+h+1
constexpr int OFF_UX = 1792;   // [8][32] u of +x faces
constexpr int OFF_UXH = 2816;  // [8][4]  u of x faces x0-4 .. x0-1
constexpr int OFF_UY = 2944;   // [8][32] u of +y faces
constexpr int OFF_UYH = 3968;  // [2][32] u of y faces of rows y0-2, y0-1
constexpr int OFF_UZ = 4224;   // [8][32] u of +z faces
constexpr int OFF_THN = 5248;  // [8][32] theta^n
constexpr int SLOT = 6272;
constexpr long long WAIT_LIMIT = 1LL << 22;  // try_wait polls before giving up

struct TParams {
  const float *x;  // plain loads of the z neighbours
  const float *u;
  float *y;
  int nx, ny, nz;
  int act_x, act_y, act_z;
  int bx_u, by_u, bz_u;  // u_f block of each axis
  long long uz_off;
  float cx, cy, cz, a, b;
  int tiles_x, tiles_y, zchunk;
  int *status;
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

template <int LIM>
__device__ __forceinline__ float flux(float u, float thC, float a, float b, bool sp) {
  return face_flux(u, limited_face<float, LIM>(thC, a, b, sp));
}

template <int LIM, int SEED>
__global__ void __launch_bounds__(TX *TY) k_struct_stage_tma(
    const TParams p, const __grid_constant__ CUtensorMap m_th,
    const __grid_constant__ CUtensorMap m_thx, const __grid_constant__ CUtensorMap m_thy,
    const __grid_constant__ CUtensorMap m_u, const __grid_constant__ CUtensorMap m_ux,
    const __grid_constant__ CUtensorMap m_uy, const __grid_constant__ CUtensorMap m_thn) {
  using F = FT<float>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[RING];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  int bid = blockIdx.x;
  const int bx = bid % p.tiles_x;
  bid /= p.tiles_x;
  const int by = bid % p.tiles_y;
  const int bz = bid / p.tiles_y;
  const int x0 = bx * TX, y0 = by * TY;
  const int z0 = bz * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const int L = z1 - z0;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int w = min(TX, nx - x0), h = min(TY, ny - y0);
  const bool valid = tx < w && ty < h;
  const bool ax = p.act_x, ay = p.act_y, az = p.act_z;

  // ---- producer: plane q (relative to z0) into slot q % RING
  auto issue = [&](int q) {
    const int slot = q % RING;
    unsigned char *s = smem + slot * SLOT;
    uint64_t *bar = &bars[slot];
    const int pz = z0 + q;
    uint32_t bytes = 1024;
    if (ax) bytes += 256 + 1024 + 128;
    if (ay) bytes += 512 + 1024 + 256;
    if (az) bytes += 1024;
    if (SEED == 1) bytes += 1024;
    // the slot was last read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(bar, bytes);
    tma3(s + OFF_TH, &m_th, bar, x0, y0, pz);
    if (ax) {
      tma3(s + OFF_XL, &m_thx, bar, wrapv(x0 - 4, nx), y0, pz);
      tma3(s + OFF_XR, &m_thx, bar, wrapv(x0 + w, nx), y0, pz);
      tma4(s + OFF_UX, &m_u, bar, x0, y0, pz, p.bx_u);
      tma4(s + OFF_UXH, &m_ux, bar, wrapv(x0 - 4, nx), y0, pz, p.bx_u);
    }
    if (ay) {
      tma3(s + OFF_YT, &m_thy, bar, x0, wrapv(y0 - 2, ny), pz);
      tma3(s + OFF_YB, &m_thy, bar, x0, wrapv(y0 + h, ny), pz);
      tma4(s + OFF_UY, &m_u, bar, x0, y0, pz, p.by_u);
      tma4(s + OFF_UYH, &m_uy, bar, x0, wrapv(y0 - 2, ny), pz, p.by_u);
    }
    if (az) tma4(s + OFF_UZ, &m_u, bar, x0, y0, pz, p.bz_u);
    if (SEED == 1) tma3(s + OFF_THN, &m_thn, bar, x0, y0, pz);
  };
  auto parity = [&](int q) { return (uint32_t)((q / RING) & 1); };
  // give up: record the timeout, wait (bounded) for the copies in flight
  auto bail = [&](int lo, int hi) {
    if (tid == 0) {
      atomicExch(p.status, (int)FL_ETIMEOUT);
      for (int q = lo; q < hi; ++q) (void)mbar_wait(&bars[q % RING], parity(q));
    }
    __syncthreads();
  };

  if (tid == 0) {
    for (int i = 0; i < RING; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = 0; q < min(RING, L); ++q) issue(q);

  // ---- z window by plain loads (column clamped for invalid threads)
  const long long plane = (long long)nx * ny;
  const long long col = (long long)min(x0 + tx, nx - 1) + (long long)nx * min(y0 + ty, ny - 1);
  auto X = [&](int k) { return p.x[col + plane * wrapv(k, nz)]; };
  float th0 = X(z0), thp1 = 0.f, thp2 = 0.f, pf = 0.f, dz_m1 = 0.f, dz_0 = 0.f, fz_prev = 0.f;
  if (az) {
    const float tm2 = X(z0 - 2), tm1 = X(z0 - 1);
    thp1 = X(z0 + 1);
    thp2 = X(z0 + 2);
    pf = X(z0 + 3);
    const float d_m2 = F::sub(tm1, tm2);
    dz_m1 = F::sub(th0, tm1);
    dz_0 = F::sub(thp1, th0);
    const float uzm = p.u[p.uz_off + col + plane * wrapv(z0 - 1, nz)];
    const bool sp = upwind_positive(uzm);
    fz_prev = flux<LIM>(uzm, sp ? tm1 : th0, dz_m1, sp ? d_m2 : dz_0, sp);
  }
  {
    const bool ok = (L > 0) ? mbar_wait(&bars[0], 0) : true;
    if (__syncthreads_or(!ok)) {
      bail(0, min(RING, L));
      return;
    }
  }

  for (int q = 0; q < L; ++q) {
    const int k = z0 + q;
    const unsigned char *s = smem + (q % RING) * SLOT;
    const float *sth = reinterpret_cast<const float *>(s + OFF_TH);
    // next z neighbour two planes ahead (plain load, used next iteration)
    float pf_next = 0.f;
    if (az && q + 1 < L) pf_next = X(k + 4);
    float acc;
    if (SEED == 0) acc = th0;
    else if (SEED == 1)
      acc = F::fma(p.a, reinterpret_cast<const float *>(s + OFF_THN)[ty * TX + tx], F::mul(p.b, th0));
    else acc = 0.f;
    if (ax) {
      const float *xl = reinterpret_cast<const float *>(s + OFF_XL) + ty * 4;
      const float *xr = reinterpret_cast<const float *>(s + OFF_XR) + ty * 4;
      const float *row = sth + ty * TX;
      float t[5];
#pragma unroll
      for (int d = -2; d <= 2; ++d) {
        const int c = tx + d;
        t[d + 2] = (c < 0) ? xl[4 + c] : ((c < w) ? row[c] : xr[min(c - w, 3)]);
      }
      const float *ux = reinterpret_cast<const float *>(s + OFF_UX) + ty * TX;
      const float up = ux[tx];
      const float um = (tx > 0) ? ux[tx - 1] : reinterpret_cast<const float *>(s + OFF_UXH)[ty * 4 + 3];
      const float dm2 = F::sub(t[1], t[0]), dm1 = F::sub(t[2], t[1]);
      const float d0 = F::sub(t[3], t[2]), dp1 = F::sub(t[4], t[3]);
      const bool spm = upwind_positive(um), spp = upwind_positive(up);
      const float fm = flux<LIM>(um, spm ? t[1] : t[2], dm1, spm ? dm2 : d0, spm);
      const float fp = flux<LIM>(up, spp ? t[2] : t[3], d0, spp ? dm1 : dp1, spp);
      acc = F::fma(-p.cx, fp, acc);
      acc = F::fma(p.cx, fm, acc);
    }
    if (ay) {
      const float *yt = reinterpret_cast<const float *>(s + OFF_YT);
      const float *yb = reinterpret_cast<const float *>(s + OFF_YB);
      float t[5];
#pragma unroll
      for (int d = -2; d <= 2; ++d) {
        const int r = ty + d;
        t[d + 2] = (r < 0) ? yt[(2 + r) * TX + tx]
                           : ((r < h) ? sth[r * TX + tx] : yb[min(r - h, 1) * TX + tx]);
      }
      const float *uy = reinterpret_cast<const float *>(s + OFF_UY);
      const float up = uy[ty * TX + tx];
      const float um = (ty > 0) ? uy[(ty - 1) * TX + tx]
                                : reinterpret_cast<const float *>(s + OFF_UYH)[TX + tx];
      const float dm2 = F::sub(t[1], t[0]), dm1 = F::sub(t[2], t[1]);
      const float d0 = F::sub(t[3], t[2]), dp1 = F::sub(t[4], t[3]);
      const bool spm = upwind_positive(um), spp = upwind_positive(up);
      const float fm = flux<LIM>(um, spm ? t[1] : t[2], dm1, spm ? dm2 : d0, spm);
      const float fp = flux<LIM>(up, spp ? t[2] : t[3], d0, spp ? dm1 : dp1, spp);
      acc = F::fma(-p.cy, fp, acc);
      acc = F::fma(p.cy, fm, acc);
    }
    float fz = 0.f, dz_p1 = 0.f;
    if (az) {
      const float uz = reinterpret_cast<const float *>(s + OFF_UZ)[ty * TX + tx];
      dz_p1 = F::sub(thp2, thp1);
      const bool sp = upwind_positive(uz);
      fz = flux<LIM>(uz, sp ? th0 : thp1, dz_0, sp ? dz_m1 : dz_p1, sp);
      acc = F::fma(-p.cz, fz, acc);
      acc = F::fma(p.cz, fz_prev, acc);
    }
    if (valid) p.y[col + plane * k] = acc;
    // rotate the z window
    if (az) {
      fz_prev = fz;
      dz_m1 = dz_0;
      dz_0 = dz_p1;
      th0 = thp1;
      thp1 = thp2;
      thp2 = pf;
      pf = pf_next;
    } else if (q + 1 < L) {
      th0 = X(k + 1);
    }
    // wait for the next plane, then let the producer refill this slot
    const bool ok = (q + 1 < L) ? mbar_wait(&bars[(q + 1) % RING], parity(q + 1)) : true;
    if (__syncthreads_or(!ok)) {
      bail(q + 1, min(q + RING, L));
      return;
    }
    if (tid == 0 && q + RING < L) issue(q + RING);
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
  k<<<grid, dim3(TX, TY), smem, st>>>(p, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5],
                                      maps[6]);
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
  if (m->kind != 0 || s.seed == 2) return false;
  if (m->nx % 4 != 0 || m->nx < 32 || m->ny < 8) return false;
  if (!m->act[0] || !m->status) return false;
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
  const cuuint32_t bmain[4] = {32, 8, 1, 1}, bx[4] = {4, 8, 1, 1}, by[4] = {32, 2, 1, 1};
  alignas(64) CUtensorMap maps[7];
  bool ok = encode(&maps[0], s.x, 3, d3, s3, bmain) && encode(&maps[1], s.x, 3, d3, s3, bx) &&
            encode(&maps[2], s.x, 3, d3, s3, by) && encode(&maps[3], s.u, 4, d4, s4, bmain) &&
            encode(&maps[4], s.u, 4, d4, s4, bx) && encode(&maps[5], s.u, 4, d4, s4, by);
  if (ok) ok = encode(&maps[6], s.seed == 1 ? s.thn : s.x, 3, d3, s3, bmain);
  if (!ok) return cudaErrorNotSupported;  // caller falls back to the plain kernel
  TParams p;
  p.x = static_cast<const float *>(s.x);
  p.u = static_cast<const float *>(s.u);
  p.y = static_cast<float *>(s.y);
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.act_x = m->act[0];
  p.act_y = m->act[1];
  p.act_z = m->act[2];
  p.bx_u = (int)(m->u_off[0] / m->C);
  p.by_u = (int)(m->u_off[1] / m->C);
  p.bz_u = (int)(m->u_off[2] / m->C);
  p.uz_off = m->u_off[2];
  const double sc = (s.seed == 0) ? s.dt : s.b * s.dt;
  p.cx = (float)(sc / m->hx);
  p.cy = (float)(sc / m->hy);
  p.cz = (float)(sc / m->hz);
  p.a = (float)s.a;
  p.b = (float)s.b;
  p.tiles_x = (nx + TX - 1) / TX;
  p.tiles_y = (ny + TY - 1) / TY;
  const long long cols = (long long)p.tiles_x * p.tiles_y;
  // about four waves of resident CTAs: zchunk = nz / ceil(4 * resident / cols)
  static int resident = 0;
  if (resident == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_struct_stage_tma<LIM_SUPERBEE, 1>,
                                                  TX * TY, RING * SLOT);
    resident = sms * (per > 0 ? per : 1);
  }
  long long nch = (4LL * resident + cols - 1) / cols;
  if (nch > nz) nch = nz;
  if (nch < 1) nch = 1;
  int zchunk = (int)((nz + nch - 1) / nch);
  if (zchunk < 8) zchunk = (nz < 8) ? nz : 8;
  p.zchunk = zchunk;
  p.status = m->status;
  const unsigned grid = (unsigned)(cols * ((nz + zchunk - 1) / zchunk));
  return s.seed == 0 ? launch_lim<0>(lim, p, maps, grid, st) : launch_lim<1>(lim, p, maps, grid, st);
}

}  // namespace fl
