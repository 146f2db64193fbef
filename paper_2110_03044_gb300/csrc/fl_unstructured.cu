// fl_unstructured.cu -- face-based meshes: validation, upstream-cell tables,
// locality renumbering, and the fused block-local stage kernel.
//
// Method (Valle et al., Section 3.1 and Algorithm 3): the upstream difference
// of face f, with upwind cell C, is the n_f-projected sum over the other faces
// j of C of their differences, orientation-corrected by the velocity sign:
//   d_U = s sum_{j in dC, j != f} (n_f . n_j) (theta_{j,c1} - theta_{j,c0}).
// On hexahedral meshes every face j of C other than the one opposite f has
// n_f . n_j = 0, and the opposite one has n_f . n_j = +-1, so the sum has a
// single term: d_U = sigma (theta_C - theta_U) with U the cell across the
// opposite face and sigma = +-1 fixed by the mesh.  mesh creation resolves U
// and sigma for both flow directions of every face, so the kernel gathers
// three cell values per face: theta_c0, theta_c1 and theta_U.
//
// Meshes of other polyhedra (tetrahedra, prisms, mixed) have faces without a
// single opposite face; for them mesh creation stores, per face and flow
// direction, every other face j of the upwind cell with n_f . n_j != 0 as a
// pair (the cell across j, coefficient (n_f . n_j) eps_j), eps_j = +1 when
// C is c0 of j, so that s d_U = sum_j coef_j (theta_j - theta_C), and the
// kernel sums it.  Non-uniform meshes (given face distances) take this
// stencil on any cell shape, with Algorithm 3's weights d_f / d_j folded
// into the coefficients; a hexahedral cell then keeps one term per face.
//
// Kernel: one CTA per cell block (a compact patch of cells in the internal
// numbering).  Phase 1 evaluates every face of the block's list once --
// upwind selection, limited theta_f and the flux u_f A_f theta_f -- into
// shared memory; phase 2 gives each cell the signed sum of its faces' fluxes
// (gather, no atomics) fused with the RK stage combination.  Faces on a block
// boundary are evaluated by both blocks from the same inputs with the same
// code, so both cells see the same flux and the scheme stays conservative.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "fl_face.cuh"
#include "fl_internal.h"
#include "fl_kernels.h"
#include "fl_unstructured.h"

namespace fl {

namespace {

constexpr int UTHREADS = 256;
constexpr unsigned SIGMA_BIT = 0x80000000u;

// ================================================================ kernels
template <class T>
struct UParams {
  const T *x;
  const T *thn;
  T *y;
  T *thf;
  const T *u;
  const int32_t *blk_cell;
  const int32_t *blk_entry;
  const int32_t *ent_face;
  const int4 *ent_cells;
  const uint16_t *slots;
  const T *area;
  const T *inv_vol;
  T a, b, bdt;  // RK combination a*thn + b*x and b*dt (times the velocity factor)
  T g;          // PRE: velocity factor of the stage
  unsigned long long flip;  // sign mask toggled into u_f before the upwind test
  const int32_t *gen_cell;  // GEN: general upstream stencil (see UnstructDev)
  const T *gen_coef;
  int kg;
  int blk0, nblk;  // the launch covers blocks [blk0, blk0 + nblk)
};

// v with its sign bit toggled when neg, on the integer pipe (opaque bits:
// otherwise the compiler may evaluate a flipped difference as both
// subtractions and a select, one FP64 add more per face entry)
template <class T>
__device__ __forceinline__ T flip_sign(T v, bool neg) {
  using F = FT<T>;
  return F::val(F::opaque_bits(v) ^ (neg ? F::SIGN : typename F::U(0)));
}

// PRE: p.u holds w_f = dt A_f u_f (pre-scaled once per call, same signs);
// phase 1 keeps theta_f and w_f of every face, and phase 2 adds w theta_f of
// each of the cell's faces with one fma -- the two flux products per face
// disappear.  The block's shared memory then holds both arrays.
// MOD (with PRE): the stage's velocity factor g is not 1 and scales the cell
// update; without it the factor is 1 and its multiply is skipped.
template <class T, int LIM, int SEED, bool PRE, bool GEN, bool MOD = false>
__global__ void __launch_bounds__(UTHREADS) k_unstruct_stage(const UParams<T> p) {
  using F = FT<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  T *s_phi = reinterpret_cast<T *>(smem);
  const int blk = p.blk0 + (int)blockIdx.x;
  const int eb = p.blk_entry[blk], ee = p.blk_entry[blk + 1];
  const int cb = p.blk_cell[blk], ce = p.blk_cell[blk + 1];
  // ---- phase 1: every face of the block once
  for (int e = eb + (int)threadIdx.x; e < ee; e += UTHREADS) {
    const int f = p.ent_face[e];
    const int4 cc = p.ent_cells[e];
    const T uf = p.u[f];
    const bool sp = upwind_positive(sign_toggled(uf, p.flip));
    const T t0 = p.x[cc.x];
    const T t1 = p.x[cc.y];
    const T tC = sp ? t0 : t1;
    const T a = F::sub(t1, t0);
    T bU;
    if (GEN) {
      // b = s d_U = sum_j coef_j (theta_j - theta_C) over the other faces of C
      const size_t base = ((size_t)f * 2 + (sp ? 0 : 1)) * (size_t)p.kg;
      bU = T(0);
      for (int k = 0; k < p.kg; ++k)
        bU = F::fma(p.gen_coef[base + k], F::sub(p.x[p.gen_cell[base + k]], tC), bU);
    } else {
      const unsigned up = sp ? (unsigned)cc.z : (unsigned)cc.w;
      const T tU = p.x[up & ~SIGMA_BIT];
      // b = s d_U = s sigma (theta_C - theta_U)
      bU = flip_sign(F::sub(tC, tU), (!sp) != ((up & SIGMA_BIT) != 0));
    }
    const T thf = limited_face<T, LIM>(tC, a, bU, sp);
    if (PRE) {
      s_phi[e - eb] = thf;
      s_phi[(ee - eb) + (e - eb)] = uf;
    } else {
      s_phi[e - eb] = F::mul(F::mul(uf, p.area[f]), thf);
    }
    if (SEED == 2 && p.thf != nullptr && cc.x >= cb && cc.x < ce) p.thf[f] = thf;
  }
  __syncthreads();
  if (PRE) {
    // phase 2 with the folded flux product: y = x - (g / V) sum sigma w theta_f
    const T *s_w = s_phi + (ee - eb);
    for (int c = cb + (int)threadIdx.x; c < ce; c += UTHREADS) {
      const uint4 sl = *reinterpret_cast<const uint4 *>(p.slots + (size_t)c * UMAXDEG);
      const unsigned w[4] = {sl.x, sl.y, sl.z, sl.w};
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 2 * 4; ++q) {
        const unsigned s16 = (w[q >> 1] >> ((q & 1) * 16)) & 0xFFFFu;
        if (s16 != 0xFFFFu) {
          const unsigned k = s16 & 0x7FFFu;
          acc = F::fma(flip_sign(s_w[k], (s16 & 0x8000u) != 0), s_phi[k], acc);
        }
      }
      const T coef = MOD ? F::mul(p.g, p.inv_vol[c]) : p.inv_vol[c];
      T out = F::fma(-coef, acc, p.x[c]);
      if (SEED == 1) out = F::fma(p.b, out, F::mul(p.a, p.thn[c]));
      p.y[c] = out;
    }
    return;
  }
  // ---- phase 2: cell sums fused with the stage update
  for (int c = cb + (int)threadIdx.x; c < ce; c += UTHREADS) {
    const uint4 sl = *reinterpret_cast<const uint4 *>(p.slots + (size_t)c * UMAXDEG);
    const unsigned w[4] = {sl.x, sl.y, sl.z, sl.w};
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 2 * 4; ++q) {
      const unsigned s16 = (w[q >> 1] >> ((q & 1) * 16)) & 0xFFFFu;
      if (s16 != 0xFFFFu) acc = F::add(acc, flip_sign(s_phi[s16 & 0x7FFFu], (s16 & 0x8000u) != 0));
    }
    // R = -acc / V
    if (SEED == 2) {
      p.y[c] = F::mul(-p.inv_vol[c], acc);
    } else {
      const T coef = F::mul(p.bdt, p.inv_vol[c]);
      T seed;
      if (SEED == 0) seed = p.x[c];
      else seed = F::fma(p.a, p.thn[c], F::mul(p.b, p.x[c]));
      p.y[c] = F::fma(-coef, acc, seed);
    }
  }
}

// w_f = (u_f A_f) dt; a product that underflows keeps the sign of u_f
__global__ void k_scale_area(const double *u, const double *area, double *w, long long nf,
                             double dt) {
  using F = FT<double>;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const double uf = u[f];
    double v = F::mul(F::mul(uf, area[f]), dt);
    if (upwind_positive(uf) && !upwind_positive(v)) v = F::val(1);
    w[f] = v;
  }
}

template <class T>
__global__ void k_unstruct_selection(const T *u, const int4 *c4, int4 *sel, long long nf) {
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const int4 cc = c4[f];
    const bool sp = upwind_positive(u[f]);
    int4 o;
    o.x = sp ? 1 : -1;
    o.y = sp ? cc.x : cc.y;
    o.z = sp ? cc.y : cc.x;
    const unsigned upv = (unsigned)(sp ? cc.z : cc.w);
    // general polyhedra: -1 unless exactly one other face of C has n_f . n_j != 0
    o.w = (upv == 0xFFFFFFFFu) ? -1 : (int)(upv & ~SIGMA_BIT);
    sel[f] = o;
  }
}

// ------------------------------------------------------------------ adjoint
// Stage adjoint on face-based meshes, as a gather (no atomics, the same
// result on every run).  The forward face value, linearised on the branch
// its evaluation takes (limited_face_lin), is
//   theta_f ~ theta_C + alpha (theta_D - theta_C) + s beta b,
// with b = sigma (theta_C - theta_U) s (hexahedra) or
// b = sum_k coef_k (theta_k - theta_C) (general polyhedra).  With
// h_f = mu_c1 / V_c1 - mu_c0 / V_c0 (the derivative of sum_c mu_c R_c with
// respect to the flux u_f A_f theta_f) and G = h_f u_f A_f, face f hands
//   C: G (1 - alpha + sigma beta)  or  G (1 - alpha - s beta sum_k coef_k),
//   D: G alpha,
//   U: -G sigma beta               or  stencil cell k: G s beta coef_k.
// A cell sums what its own faces hand it (as C or D) and what the faces
// whose upstream stencil names it hand it (the lists built by
// unstruct_adjoint_prepare), evaluating each face where it needs it.
template <class T>
struct UAParams {
  const T *x, *mu, *v1, *v2;
  T *out;
  const T *u;        // u_f, or w_f = (dt) A_f u_f when PRE
  const T *area, *inv_vol;
  const int4 *c4;
  const int32_t *gen_cell;
  const T *gen_coef;
  int kg;
  const int32_t *cf_ptr, *cf, *inv_ptr, *inv_f;
  const uint8_t *inv_sk;
  T e1, e2, b, bdt;
  int bare;
  long long c0, C;  // the cells [c0, C) are computed
};

template <class T>
struct ULin {
  T G, al, be, sumc;  // sumc: sigma (hexahedra) or sum_k coef_k (general)
  bool sp;
};

template <class T, int LIM, bool GEN, bool PRE>
__device__ __forceinline__ ULin<T> u_lin(const UAParams<T> &p, int f) {
  using F = FT<T>;
  ULin<T> r;
  const int4 cc = p.c4[f];
  const T uf = p.u[f];
  r.sp = upwind_positive(uf);
  const T t0 = p.x[cc.x], t1 = p.x[cc.y];
  const T tC = r.sp ? t0 : t1;
  const T a = F::sub(t1, t0);
  T b;
  if (GEN) {
    const size_t base = ((size_t)f * 2 + (r.sp ? 0 : 1)) * (size_t)p.kg;
    b = T(0);
    r.sumc = T(0);
    for (int k = 0; k < p.kg; ++k) {
      b = F::fma(p.gen_coef[base + k], F::sub(p.x[p.gen_cell[base + k]], tC), b);
      r.sumc = F::add(r.sumc, p.gen_coef[base + k]);
    }
  } else {
    const unsigned up = r.sp ? (unsigned)cc.z : (unsigned)cc.w;
    const bool sneg = (up & SIGMA_BIT) != 0;
    b = flip_sign(F::sub(tC, p.x[up & ~SIGMA_BIT]), (!r.sp) != sneg);
    r.sumc = sneg ? T(-1) : T(1);
  }
  T c1;
  limited_face_lin<T, LIM>(a, b, r.al, r.be, c1);
  const T h = F::sub(F::mul(p.mu[cc.y], p.inv_vol[cc.y]), F::mul(p.mu[cc.x], p.inv_vol[cc.x]));
  r.G = F::mul(h, PRE ? uf : F::mul(uf, p.area[f]));
  return r;
}

template <class T, int LIM, bool GEN, bool PRE>
__global__ void __launch_bounds__(256) k_unstruct_adjoint(const UAParams<T> p) {
  using F = FT<T>;
  for (long long c = p.c0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.C;
       c += (long long)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int q = p.cf_ptr[c]; q < p.cf_ptr[c + 1]; ++q) {
      const int f = p.cf[q];
      const ULin<T> L = u_lin<T, LIM, GEN, PRE>(p, f);
      const int4 cc = p.c4[f];
      const bool isC = L.sp ? (cc.x == c) : (cc.y == c);
      if (isC) {
        // 1 - alpha + sigma beta (hexahedra); 1 - alpha - s beta sum coef
        const T up = GEN ? F::mul(L.sp ? -L.be : L.be, L.sumc) : F::mul(L.sumc, L.be);
        acc = F::fma(L.G, F::add(F::sub(T(1), L.al), up), acc);
      } else {
        acc = F::fma(L.G, L.al, acc);
      }
    }
    for (int q = p.inv_ptr[c]; q < p.inv_ptr[c + 1]; ++q) {
      const int f = p.inv_f[q];
      const int sk = p.inv_sk[q];
      const bool side_pos = (sk & 1) == 0;  // side 0: C = c0, the s > 0 side
      if (upwind_positive(p.u[f]) != side_pos) continue;
      const ULin<T> L = u_lin<T, LIM, GEN, PRE>(p, f);
      if (GEN) {
        const T coef = p.gen_coef[((size_t)f * 2 + (sk & 1)) * (size_t)p.kg + (sk >> 1)];
        acc = F::fma(L.G, F::mul(L.sp ? L.be : -L.be, coef), acc);
      } else {
        acc = F::fma(L.G, F::mul(-L.sumc, L.be), acc);
      }
    }
    T o;
    if (p.bare) {
      o = acc;
    } else {
      o = F::fma(p.bdt, acc, F::mul(p.b, p.mu[c]));
      if (p.v1) o = F::fma(p.e1, p.v1[c], o);
      if (p.v2) o = F::fma(p.e2, p.v2[c], o);
    }
    p.out[c] = o;
  }
}

// w_f = fac A_f u_f for the adjoint (fac = dt, or 1), any precision; a
// product that underflows keeps the sign of u_f
template <class T>
__global__ void k_scale_area_t(const T *u, const T *area, T *w, long long nf, T fac) {
  using F = FT<T>;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const T uf = u[f];
    T v = F::mul(F::mul(uf, area[f]), fac);
    if (upwind_positive(uf) && !upwind_positive(v)) v = F::val(1);
    w[f] = v;
  }
}

template <class T, int SEED, bool PRE, bool GEN, bool MOD = false>
cudaError_t launch_lim(int lim, const fl_mesh *m, const UParams<T> &p, cudaStream_t st) {
  const int nb = p.nblk;
  const int ents = (p.blk0 == 0 && nb == m->u.nb_interior && nb < m->u.n_blocks)
                       ? m->u.max_entries_interior
                   : (p.blk0 > 0 && p.blk0 == m->u.nb_interior) ? m->u.max_entries_rim
                                                                : m->u.max_block_entries;
  const size_t smem = (size_t)ents * sizeof(T) * (PRE ? 2 : 1);
  if (nb == 0) return cudaSuccess;
#define FL_U_CASE(L)                                                                           \
  case L: {                                                                                    \
    auto k = k_unstruct_stage<T, L, SEED, PRE, GEN, MOD>;                                      \
    if (smem > 48 * 1024) {                                                                    \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                           (int)smem);                                         \
      if (e != cudaSuccess) return e;                                                          \
    }                                                                                          \
    k<<<nb, UTHREADS, smem, st>>>(p);                                                          \
    return cudaGetLastError();                                                                 \
  }
  switch (lim) {
    FL_U_CASE(LIM_UPWIND)
    FL_U_CASE(LIM_CENTRAL)
    FL_U_CASE(LIM_MINMOD)
    FL_U_CASE(LIM_VANLEER)
    FL_U_CASE(LIM_SUPERBEE)
    FL_U_CASE(LIM_SMART)
  }
#undef FL_U_CASE
  return cudaErrorInvalidValue;
}

template <class T, bool GEN>
cudaError_t dispatch_seed(int lim, const fl_mesh *m, const UParams<T> &p, int seed, bool pre,
                          cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (pre && p.g != T(1)) {
      if (seed == 0) return launch_lim<T, 0, true, GEN, true>(lim, m, p, st);
      return launch_lim<T, 1, true, GEN, true>(lim, m, p, st);
    }
    if (pre) {
      if (seed == 0) return launch_lim<T, 0, true, GEN>(lim, m, p, st);
      return launch_lim<T, 1, true, GEN>(lim, m, p, st);
    }
  }
  switch (seed) {
    case 0: return launch_lim<T, 0, false, GEN>(lim, m, p, st);
    case 1: return launch_lim<T, 1, false, GEN>(lim, m, p, st);
    default: return launch_lim<T, 2, false, GEN>(lim, m, p, st);
  }
}

template <class T>
cudaError_t run_ustage(const fl_mesh *m, int lim, const StageArgs &s, cudaStream_t st) {
  UParams<T> p;
  p.x = static_cast<const T *>(s.x);
  p.thn = static_cast<const T *>(s.thn);
  p.y = static_cast<T *>(s.y);
  p.thf = static_cast<T *>(s.thf);
  const bool pre = s.w != nullptr && sizeof(T) == 8 && s.seed != 2;
  p.u = static_cast<const T *>(pre ? s.w : s.u);
  p.blk_cell = m->u.blk_cell;
  p.blk_entry = m->u.blk_entry;
  p.ent_face = m->u.ent_face;
  p.ent_cells = m->u.ent_cells;
  p.slots = m->u.cell_slots;
  if (sizeof(T) == 8) {
    p.area = reinterpret_cast<const T *>(m->u.area);
    p.inv_vol = reinterpret_cast<const T *>(m->u.inv_vol);
  } else {
    p.area = reinterpret_cast<const T *>(m->u.area_f);
    p.inv_vol = reinterpret_cast<const T *>(m->u.inv_vol_f);
  }
  p.a = blend_a<T>(s.a, s.b);
  p.b = (T)s.b;
  // the flow of this stage is g u_f: fluxes scale by g, and g < 0 flips
  // every face's upwind side (the bare operator has g = 1)
  const double g = (s.seed == 2) ? 1.0 : s.g;
  p.bdt = (T)(s.b * s.dt * g);
  p.g = (T)g;
  p.flip = (g < 0) ? (sizeof(T) == 8 ? 0x8000000000000000ull : 0x80000000ull) : 0ull;
  p.kg = m->u.kg;
  p.gen_cell = m->u.gen_cell;
  p.gen_coef = (sizeof(T) == 8) ? reinterpret_cast<const T *>(m->u.gen_coef)
                                : reinterpret_cast<const T *>(m->u.gen_coef_f);
  // the blocks of the cell range: every owned cell, the interior, or the rim
  p.blk0 = 0;
  p.nblk = m->u.n_blocks;
  if (s.chi >= 0) {
    const int64_t lo = s.clo, hi = s.chi;
    const bool whole = lo == 0 && hi == m->n_owned;
    if (!whole && lo == 0 && hi == m->n_interior) {
      p.nblk = m->u.nb_interior;
    } else if (!whole && lo == m->n_interior && hi == m->n_owned) {
      p.blk0 = m->u.nb_interior;
      p.nblk = m->u.n_blocks - m->u.nb_interior;
    } else if (!whole) {
      return cudaErrorInvalidValue;  // checked by the entry point
    }
  }
  if (m->u.kg > 0) return dispatch_seed<T, true>(lim, m, p, s.seed, pre, st);
  return dispatch_seed<T, false>(lim, m, p, s.seed, pre, st);
}

// ============================================================ host build
// Run fn(begin, end) over [0, n) on the host cores (mesh set-up only).
template <class Fn>
void parallel_for(int64_t n, Fn fn) {
  unsigned nt = std::thread::hardware_concurrency();
  nt = std::max(1u, std::min(nt, 64u));
  if (n < 50000 || nt == 1) {
    fn((int64_t)0, n);
    return;
  }
  std::vector<std::thread> ts;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t a = (int64_t)t * chunk, b = std::min(n, a + chunk);
    if (a < b) ts.emplace_back(fn, a, b);
  }
  for (auto &th : ts) th.join();
}

// First error raised inside a parallel loop.
struct ErrSink {
  std::atomic<int> set{0};
  fl_status st = FL_OK;
  char msg[256] = "";
  std::mutex mu;
  void put(fl_status s, const char *fmt, long long a, long long b = 0) {
    std::lock_guard<std::mutex> lock(mu);
    if (set.load()) return;
    st = s;
    snprintf(msg, sizeof(msg), fmt, a, b);
    set.store(1);
  }
};

// Sort in parallel: chunks sorted concurrently, then merged pairwise.
template <class It, class Cmp>
void parallel_sort(It first, It last, Cmp cmp) {
  const int64_t n = last - first;
  unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  if (n < 200000 || nt == 1) {
    std::sort(first, last, cmp);
    return;
  }
  std::vector<int64_t> cut;
  for (unsigned t = 0; t <= nt; ++t) cut.push_back(n * (int64_t)t / nt);
  {
    std::vector<std::thread> ts;
    for (unsigned t = 0; t < nt; ++t)
      ts.emplace_back([&, t] { std::sort(first + cut[t], first + cut[t + 1], cmp); });
    for (auto &th : ts) th.join();
  }
  while (cut.size() > 2) {
    std::vector<int64_t> next;
    std::vector<std::thread> ts;
    for (size_t i = 0; i + 2 < cut.size(); i += 2) {
      ts.emplace_back([&, i] {
        std::inplace_merge(first + cut[i], first + cut[i + 1], first + cut[i + 2], cmp);
      });
      next.push_back(cut[i]);
    }
    if (cut.size() % 2 == 0) next.push_back(cut[cut.size() - 2]);
    next.push_back(cut.back());
    for (auto &th : ts) th.join();
    cut.swap(next);
  }
}

template <class V>
fl_status upload(const std::vector<V> &h, V **d) {
  *d = nullptr;
  if (h.empty()) return FL_OK;
  if (cudaMalloc(reinterpret_cast<void **>(d), h.size() * sizeof(V)) != cudaSuccess)
    return fail(FL_ENOMEM, "device allocation of %zu bytes failed", h.size() * sizeof(V));
  if (cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(FL_ECUDA, "host-to-device copy failed");
  return FL_OK;
}

struct HostMesh {
  int64_t C = 0, F = 0;
  std::vector<int32_t> c0, c1;
  std::vector<double> n;  // [F][3]
  std::vector<int64_t> cf_ptr;
  std::vector<int32_t> cf_idx;
  std::vector<int32_t> up[2];  // upstream cell per face and side (side 0: C = c0)
  std::vector<int8_t> sig[2];  // sigma per face and side
};

inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Direction classes of the face normals (at most three mutually orthogonal
// directions on a Cartesian-like hexahedral mesh).  Returns false otherwise.
bool direction_classes(const HostMesh &h, std::vector<int8_t> &cls, std::vector<int8_t> &sgn) {
  std::vector<std::array<double, 3>> dirs;
  cls.assign(h.F, 0);
  sgn.assign(h.F, 1);
  for (int64_t f = 0; f < h.F; ++f) {
    const double *nf = &h.n[3 * f];
    int k = -1;
    for (size_t q = 0; q < dirs.size(); ++q) {
      const double d = dot3(nf, dirs[q].data());
      if (std::fabs(d) > 0.9) {
        k = (int)q;
        sgn[f] = d > 0 ? 1 : -1;
        break;
      }
    }
    if (k < 0) {
      if (dirs.size() == 3) return false;
      dirs.push_back({nf[0], nf[1], nf[2]});
      k = (int)dirs.size() - 1;
      sgn[f] = 1;
    }
    cls[f] = (int8_t)k;
  }
  return true;
}

// Internal cell order.  On Cartesian-like meshes the cells get integer
// lattice coordinates by a breadth-first walk along the face normals and are
// sorted into 8x8x8 tiles (each tile becomes one block).  Otherwise blocks are
// grown greedily as breadth-first balls of up to UBLOCK cells.
void renumber_cells(const HostMesh &h, std::vector<int32_t> &order, std::vector<int32_t> &blk_cell) {
  const int64_t C = h.C;
  std::vector<int8_t> cls, sgn;
  order.clear();
  blk_cell.clear();
  if (direction_classes(h, cls, sgn)) {
    std::vector<int64_t> key(C, -1);
    std::vector<int32_t> cx(C), cy(C), cz(C), comp(C, -1);
    int ncomp = 0;
    std::vector<int32_t> queue;
    queue.reserve(C);
    for (int64_t s = 0; s < C; ++s) {
      if (comp[s] >= 0) continue;
      comp[s] = ncomp;
      cx[s] = cy[s] = cz[s] = 0;
      queue.clear();
      queue.push_back((int32_t)s);
      for (size_t qi = 0; qi < queue.size(); ++qi) {
        const int32_t c = queue[qi];
        for (int64_t t = h.cf_ptr[c]; t < h.cf_ptr[c + 1]; ++t) {
          const int32_t f = h.cf_idx[t];
          const bool is0 = (h.c0[f] == c);
          const int32_t nb = is0 ? h.c1[f] : h.c0[f];
          if (comp[nb] >= 0) continue;
          const int step = (is0 ? 1 : -1) * sgn[f];
          comp[nb] = ncomp;
          cx[nb] = cx[c] + (cls[f] == 0 ? step : 0);
          cy[nb] = cy[c] + (cls[f] == 1 ? step : 0);
          cz[nb] = cz[c] + (cls[f] == 2 ? step : 0);
          queue.push_back(nb);
        }
      }
      ++ncomp;
    }
    // sort by (component, tile z, tile y, tile x) and, inside a tile, by
    // (z, y, x): one packed 64-bit tile key plus a 9-bit in-tile index
    auto fdiv = [](int32_t v) { return (v >= 0) ? v / 8 : -((-v + 7) / 8); };
    int32_t lo[3] = {0, 0, 0};
    for (int64_t c = 0; c < C; ++c) {
      lo[0] = std::min(lo[0], fdiv(cx[c]));
      lo[1] = std::min(lo[1], fdiv(cy[c]));
      lo[2] = std::min(lo[2], fdiv(cz[c]));
    }
    struct K {
      uint64_t tile;
      uint32_t in_tile;
      int32_t c;
    };
    std::vector<K> ks(C);
    for (int64_t c = 0; c < C; ++c) {
      const uint64_t tx = (uint64_t)(fdiv(cx[c]) - lo[0]);
      const uint64_t ty = (uint64_t)(fdiv(cy[c]) - lo[1]);
      const uint64_t tz = (uint64_t)(fdiv(cz[c]) - lo[2]);
      // components < 2^13, tile coordinates < 2^17 each
      const uint64_t key = ((uint64_t)comp[c] << 51) | (tz << 34) | (ty << 17) | tx;
      const uint32_t loc = (uint32_t)(((cz[c] & 7) << 6) | ((cy[c] & 7) << 3) | (cx[c] & 7));
      ks[c] = {key, loc, (int32_t)c};
    }
    parallel_sort(ks.begin(), ks.end(), [](const K &a, const K &b) {
      return a.tile != b.tile ? a.tile < b.tile : a.in_tile < b.in_tile;
    });
    order.resize(C);
    blk_cell.push_back(0);
    for (int64_t i = 0; i < C; ++i) {
      order[i] = ks[i].c;
      if (i > 0 && (ks[i].tile != ks[i - 1].tile || i - blk_cell.back() >= UBLOCK))
        blk_cell.push_back((int32_t)i);
    }
    blk_cell.push_back((int32_t)C);
    return;
  }
  // greedy breadth-first balls
  std::vector<uint8_t> taken(C, 0);
  std::vector<int32_t> q;
  blk_cell.push_back(0);
  int64_t next_seed = 0;
  while ((int64_t)order.size() < C) {
    while (taken[next_seed]) ++next_seed;
    q.clear();
    q.push_back((int32_t)next_seed);
    taken[next_seed] = 1;
    size_t qi = 0;
    int count = 0;
    while (qi < q.size() && count < UBLOCK) {
      const int32_t c = q[qi++];
      order.push_back(c);
      ++count;
      for (int64_t t = h.cf_ptr[c]; t < h.cf_ptr[c + 1]; ++t) {
        const int32_t f = h.cf_idx[t];
        const int32_t nb = (h.c0[f] == c) ? h.c1[f] : h.c0[f];
        if (!taken[nb]) {
          taken[nb] = 1;
          q.push_back(nb);
        }
      }
    }
    for (size_t r = qi; r < q.size(); ++r) taken[q[r]] = 0;  // not placed yet
    blk_cell.push_back((int32_t)order.size());
  }
}

}  // namespace

// ----------------------------------------------------------------- create
fl_status unstruct_create(int64_t C, int64_t F, const int32_t *face_cells, const double *normals,
                          const double *areas, const double *volumes, const double *distances,
                          unsigned flags, int64_t n_owned, int64_t n_interior, fl_mesh **out) {
  if (C < 0 || F < 0) return fail(FL_EINVAL, "negative size");
  // a local mesh of a partition updates cells [0, n_owned) only
  const bool local = n_owned < C || n_interior < n_owned;
  if (C >= (1LL << 31) - 1 || F >= (1LL << 31) - 1) return fail(FL_EUNSUPPORTED, "sizes must be < 2^31");
  if ((F > 0 && (!face_cells || !normals || !areas)) || (C > 0 && !volumes))
    return fail(FL_EINVAL, "NULL input array");
  if (flags & ~FL_RENUMBER) return fail(FL_EINVAL, "unknown flags 0x%x", flags);
  HostMesh h;
  h.C = C;
  h.F = F;
  h.c0.resize(F);
  h.c1.resize(F);
  h.n.assign(normals, normals + 3 * F);
  ErrSink err;
  parallel_for(F, [&](int64_t lo, int64_t hi) {
    for (int64_t f = lo; f < hi && !err.set.load(); ++f) {
      const int32_t a = face_cells[2 * f], b = face_cells[2 * f + 1];
      if (a < 0 || b < 0 || a >= C || b >= C)
        return err.put(FL_EINDEX, "face %lld: cell index out of range", f);
      if (a == b) return err.put(FL_EINVAL, "face %lld: c0 == c1", f);
      const double *nf = &normals[3 * f];
      if (!(std::fabs(dot3(nf, nf) - 1.0) < 1e-9))
        return err.put(FL_EINVAL, "face %lld: normal is not unit", f);
      if (!(areas[f] > 0) || !std::isfinite(areas[f]))
        return err.put(FL_EINVAL, "face %lld: bad area", f);
      if (distances && (!(distances[f] > 0) || !std::isfinite(distances[f])))
        return err.put(FL_EINVAL, "face %lld: bad distance", f);
      h.c0[f] = a;
      h.c1[f] = b;
    }
  });
  parallel_for(C, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi && !err.set.load(); ++c)
      if (!(volumes[c] > 0) || !std::isfinite(volumes[c]))
        return err.put(FL_EINVAL, "cell %lld: bad volume", c);
  });
  if (err.set.load()) return fail(err.st, "%s", err.msg);
  // cell -> faces (each list in ascending face id)
  h.cf_ptr.assign(C + 1, 0);
  for (int64_t f = 0; f < F; ++f) {
    h.cf_ptr[h.c0[f] + 1]++;
    h.cf_ptr[h.c1[f] + 1]++;
  }
  for (int64_t c = 0; c < C; ++c) {
    if (h.cf_ptr[c + 1] > UMAXDEG)
      return fail(FL_EUNSUPPORTED, "cell %lld has %lld faces (at most %d)", (long long)c,
                  (long long)h.cf_ptr[c + 1], UMAXDEG);
    h.cf_ptr[c + 1] += h.cf_ptr[c];
  }
  h.cf_idx.resize(h.cf_ptr[C]);
  {
    std::vector<int64_t> fill(h.cf_ptr.begin(), h.cf_ptr.end() - 1);
    for (int64_t f = 0; f < F; ++f) {
      h.cf_idx[fill[h.c0[f]]++] = (int32_t)f;
      h.cf_idx[fill[h.c1[f]]++] = (int32_t)f;
    }
  }
  // The cells whose upstream stencil is resolved: every cell of a whole
  // mesh; in a local mesh the owned cells and the halo cells next to them
  // (the upwind cell of a face of an owned cell is one of these, and the
  // caller gives them all their faces).  The outer halo cells only supply
  // values: their face lists may be cut, and no face evaluated for an owned
  // cell has one of them upwind.
  std::vector<uint8_t> resolve(C, local ? 0 : 1);
  if (local) {
    for (int64_t c = 0; c < n_owned; ++c) {
      resolve[c] = 1;
      for (int64_t t = h.cf_ptr[c]; t < h.cf_ptr[c + 1]; ++t) {
        const int32_t f = h.cf_idx[t];
        resolve[h.c0[f]] = 1;
        resolve[h.c1[f]] = 1;
      }
    }
  }
  // duplicate faces (same cell pair and the same oriented normal), then the
  // upstream cell and sign for both flow directions of every face, cell by
  // cell: for each face f of cell C, the one other face j of C with
  // n_f . n_j = +-1 (all others must be orthogonal to f)
  for (int side = 0; side < 2; ++side) {
    h.up[side].assign(F, -1);
    h.sig[side].assign(F, 0);
  }
  std::atomic<bool> general(false);
  parallel_for(C, [&](int64_t lo, int64_t hi) {
    double nrm[UMAXDEG][3];
    int32_t fl_[UMAXDEG];
    for (int64_t Cc = lo; Cc < hi && !err.set.load(); ++Cc) {
      if (!resolve[Cc]) continue;
      const int deg = (int)(h.cf_ptr[Cc + 1] - h.cf_ptr[Cc]);
      for (int a = 0; a < deg; ++a) {
        fl_[a] = h.cf_idx[h.cf_ptr[Cc] + a];
        for (int d = 0; d < 3; ++d) nrm[a][d] = h.n[3 * (int64_t)fl_[a] + d];
      }
      for (int a = 0; a < deg; ++a)
        for (int b = a + 1; b < deg; ++b) {
          const int32_t f = fl_[a], g = fl_[b];
          const double w = dot3(nrm[a], nrm[b]);
          const bool same = (h.c0[f] == h.c0[g] && h.c1[f] == h.c1[g] && w > 0.999) ||
                            (h.c0[f] == h.c1[g] && h.c1[f] == h.c0[g] && w < -0.999);
          if (same) return err.put(FL_EINVAL, "faces %lld and %lld are the same face", f, g);
        }
      for (int a = 0; a < deg; ++a) {
        const int32_t f = fl_[a];
        int found = 0, bstar = -1;
        double wstar = 0;
        for (int b = 0; b < deg; ++b) {
          if (b == a) continue;
          const double w = dot3(nrm[a], nrm[b]);
          if (std::fabs(w) > 0.5) {
            ++found;
            bstar = b;
            wstar = w;
          } else if (std::fabs(w) > 1e-9) {
            found = -1;  // neither parallel nor orthogonal: a general polyhedron
            break;
          }
        }
        if (found != 1 || std::fabs(std::fabs(wstar) - 1.0) > 1e-9) {
          general.store(true);
          continue;
        }
        const int32_t j = fl_[bstar];
        // side 0: C is c0 of f (flow c0 -> c1); side 1: C is c1 of f
        const int side = (h.c0[f] == Cc) ? 0 : 1;
        const bool jc1 = (h.c1[j] == Cc);
        h.up[side][f] = jc1 ? h.c0[j] : h.c1[j];
        // d_U = s w (theta_{j,c1} - theta_{j,c0}) = sigma (theta_C - theta_U)
        const int sgn = side == 0 ? 1 : -1;
        const int w = wstar > 0 ? 1 : -1;
        h.sig[side][f] = (int8_t)(sgn * w * (jc1 ? 1 : -1));
      }
    }
  });
  if (err.set.load()) return fail(err.st, "%s", err.msg);
  // Face distances (non-uniform spacing, Algorithm 3) weight every term of
  // the upstream stencil by d_f / d_j; they take the general stencil, whose
  // coefficients carry the weights, on any cell shape.
  if (distances && F > 0) general.store(true);
  // ---- general polyhedra: the weighted upstream stencil of every face and
  // side (the oracle's definition: all other faces j of C, weight n_f . n_j,
  // times d_f / d_j when distances are given).  Only the terms with a
  // nonzero weight are stored, in the cell's face order: a face orthogonal to
  // f adds nothing, so a hexahedral cell keeps one term (its opposite face)
  // and a prism's quadrilateral faces drop their orthogonal neighbours.
  int kg = 0;
  std::vector<int32_t> gcell;
  std::vector<double> gcoef;
  if (general.load()) {
    std::atomic<int> kmax(1);
    parallel_for(F, [&](int64_t lo, int64_t hi) {
      int local = 1;
      for (int64_t f = lo; f < hi; ++f)
        for (int side = 0; side < 2; ++side) {
          const int32_t Cc = side == 0 ? h.c0[f] : h.c1[f];
          if (!resolve[Cc]) continue;
          int nz = 0;
          for (int64_t q = h.cf_ptr[Cc]; q < h.cf_ptr[Cc + 1]; ++q) {
            const int32_t j = h.cf_idx[q];
            if (j != f && dot3(&h.n[3 * f], &h.n[3 * (int64_t)j]) != 0.0) ++nz;
          }
          local = std::max(local, nz);
        }
      int cur = kmax.load();
      while (local > cur && !kmax.compare_exchange_weak(cur, local)) {
      }
    });
    kg = kmax.load();
    gcell.assign((size_t)F * 2 * kg, 0);
    gcoef.assign((size_t)F * 2 * kg, 0.0);
    parallel_for(F, [&](int64_t lo, int64_t hi) {
      for (int64_t f = lo; f < hi; ++f)
        for (int side = 0; side < 2; ++side) {
          const int32_t Cc = side == 0 ? h.c0[f] : h.c1[f];
          const size_t base = ((size_t)f * 2 + side) * kg;
          int k = 0;
          int32_t U = -1;
          for (int64_t q = h.cf_ptr[Cc]; q < h.cf_ptr[Cc + 1] && resolve[Cc]; ++q) {
            const int32_t j = h.cf_idx[q];
            if (j == f) continue;
            const double w = dot3(&h.n[3 * f], &h.n[3 * (int64_t)j]);
            if (w == 0.0) continue;
            const bool c_is_c0 = (h.c0[j] == Cc);
            const int32_t other = c_is_c0 ? h.c1[j] : h.c0[j];
            gcell[base + k] = other;
            const double wd = distances ? w * (distances[f] / distances[j]) : w;
            gcoef[base + k] = c_is_c0 ? wd : -wd;
            ++k;
            U = other;
          }
          h.up[side][f] = (k == 1) ? U : -1;
          for (; k < kg; ++k) gcell[base + k] = Cc;  // coef 0: no contribution
          h.sig[side][f] = 1;
        }
    });
  }
  // ---- internal numbering
  std::vector<int32_t> order, blk_cell;
  const bool renum = (flags & FL_RENUMBER) != 0;
  int nb_interior = 0;
  if (local) {
    // blocks cover the interior cells, then the rim cells, never both, and
    // no halo cell.  With FL_RENUMBER the interior and the rim each take the
    // order of the whole local mesh's renumbering (compact tiles or balls);
    // the halo cells keep the caller's order (a neighbour's values arrive as
    // one slice).  Otherwise the caller's order.
    std::vector<int32_t> full, full_blk;
    if (renum && C > 0) {
      renumber_cells(h, full, full_blk);
    } else {
      full.resize(C);
      std::iota(full.begin(), full.end(), 0);
      for (int64_t c = 0; c <= C; c += UBLOCK) full_blk.push_back((int32_t)c);
      if (full_blk.back() != C) full_blk.push_back((int32_t)C);
    }
    order.clear();
    order.reserve(C);
    blk_cell.clear();
    // interior: a new block where the whole-mesh order starts one (a tile)
    // or after UBLOCK cells, so the interior's blocks stay whole tiles
    // where no rim cell was taken out
    {
      size_t b = 0;
      int64_t prev = -1, count = 0;
      for (int64_t i = 0; i < C; ++i) {
        while (b + 1 < full_blk.size() && full_blk[b + 1] <= i) ++b;
        const int32_t c = full[i];
        if (c >= n_interior) continue;
        if ((int64_t)b != prev || count == UBLOCK) {
          blk_cell.push_back((int32_t)order.size());
          prev = (int64_t)b;
          count = 0;
        }
        order.push_back(c);
        ++count;
      }
    }
    nb_interior = (int)blk_cell.size();
    // rim cells lie in a thin shell: runs of them are scattered in space, so
    // their blocks are kept small (fewer faces per block, less shared memory)
    for (int64_t i = 0; i < C; ++i) {
      const int32_t c = full[i];
      if (c < n_interior || c >= n_owned) continue;
      if ((order.size() - (size_t)n_interior) % (UBLOCK / 4) == 0)
        blk_cell.push_back((int32_t)order.size());
      order.push_back(c);
    }
    for (int64_t c = n_owned; c < C; ++c) order.push_back((int32_t)c);
    blk_cell.push_back((int32_t)n_owned);
  } else if (renum && C > 0) {
    renumber_cells(h, order, blk_cell);
  } else {
    order.resize(C);
    std::iota(order.begin(), order.end(), 0);
    blk_cell.clear();
    for (int64_t c = 0; c < C; c += UBLOCK) blk_cell.push_back((int32_t)c);
    blk_cell.push_back((int32_t)C);
  }
  if (!local) nb_interior = (int)blk_cell.size() - 1;
  std::vector<int32_t> cell_new(C);
  for (int64_t i = 0; i < C; ++i) cell_new[order[i]] = (int32_t)i;
  // faces: by the lower internal cell, then by user id (a stable counting
  // sort on the owner cell)
  std::vector<int32_t> face_order(F);
  if (renum) {
    std::vector<int64_t> cnt(C + 1, 0);
    std::vector<int32_t> owner(F);
    for (int64_t f = 0; f < F; ++f) {
      owner[f] = std::min(cell_new[h.c0[f]], cell_new[h.c1[f]]);
      cnt[owner[f] + 1]++;
    }
    for (int64_t c = 0; c < C; ++c) cnt[c + 1] += cnt[c];
    for (int64_t f = 0; f < F; ++f) face_order[cnt[owner[f]]++] = (int32_t)f;
  } else {
    std::iota(face_order.begin(), face_order.end(), 0);
  }
  std::vector<int32_t> face_new(F);
  for (int64_t i = 0; i < F; ++i) face_new[face_order[i]] = (int32_t)i;
  // per-face records in internal numbering
  std::vector<int4> c4(F);
  std::vector<double> area_i(F), vol_i(C), ivol_i(C);
  parallel_for(F, [&](int64_t lo, int64_t hi) {
  for (int64_t f = lo; f < hi; ++f) {
    const int32_t fi = face_new[f];
    int4 r;
    r.x = cell_new[h.c0[f]];
    r.y = cell_new[h.c1[f]];
    // (general polyhedra: the single upstream cell where one exists, else -1;
    // the kernel reads the weighted stencil instead)
    r.z = h.up[0][f] < 0 ? -1
                         : (int)((unsigned)cell_new[h.up[0][f]] | (h.sig[0][f] < 0 ? SIGMA_BIT : 0u));
    r.w = h.up[1][f] < 0 ? -1
                         : (int)((unsigned)cell_new[h.up[1][f]] | (h.sig[1][f] < 0 ? SIGMA_BIT : 0u));
    c4[fi] = r;
    area_i[fi] = areas[f];
  }
  });
  for (int64_t c = 0; c < C; ++c) {
    vol_i[cell_new[c]] = volumes[c];
    ivol_i[cell_new[c]] = 1.0 / volumes[c];
  }
  // internal cell -> internal faces
  std::vector<int64_t> icf_ptr(C + 1, 0);
  for (int64_t f = 0; f < F; ++f) {
    icf_ptr[c4[f].x + 1]++;
    icf_ptr[c4[f].y + 1]++;
  }
  for (int64_t c = 0; c < C; ++c) icf_ptr[c + 1] += icf_ptr[c];
  std::vector<int32_t> icf(icf_ptr[C]);
  {
    std::vector<int64_t> fill(icf_ptr.begin(), icf_ptr.end() - 1);
    for (int64_t f = 0; f < F; ++f) {
      icf[fill[c4[f].x]++] = (int32_t)f;
      icf[fill[c4[f].y]++] = (int32_t)f;
    }
  }
  // block entry lists and per-cell slots: blocks are independent, so the
  // lists are built in parallel (count, prefix sum, fill)
  const int nb = (int)blk_cell.size() - 1;
  std::vector<int32_t> blk_entry(nb + 1, 0);
  std::vector<uint16_t> slots((size_t)C * UMAXDEG, 0xFFFF);
  auto block_list = [&](int b, std::vector<int32_t> &list) {
    const int32_t cb = blk_cell[b], ce = blk_cell[b + 1];
    list.clear();
    for (int32_t c = cb; c < ce; ++c)
      for (int64_t t = icf_ptr[c]; t < icf_ptr[c + 1]; ++t) {
        const int32_t f = icf[t];
        const int32_t o = (c4[f].x == c) ? c4[f].y : c4[f].x;
        // a face inside the block is listed once (from its lower cell)
        if (o >= cb && o < ce && o < c) continue;
        list.push_back(f);
      }
    std::sort(list.begin(), list.end());
  };
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    std::vector<int32_t> list;
    for (int64_t b = lo; b < hi; ++b) {
      block_list((int)b, list);
      blk_entry[b + 1] = (int32_t)list.size();
    }
  });
  int max_entries = 0, max_int = 0, max_rim = 0;
  for (int b = 0; b < nb; ++b) {
    if (blk_entry[b + 1] > 0x7FFF)
      return fail(FL_EUNSUPPORTED, "block %d has %d faces", b, blk_entry[b + 1]);
    max_entries = std::max(max_entries, (int)blk_entry[b + 1]);
    if (b < nb_interior) max_int = std::max(max_int, (int)blk_entry[b + 1]);
    else max_rim = std::max(max_rim, (int)blk_entry[b + 1]);
    blk_entry[b + 1] += blk_entry[b];
  }
  std::vector<int32_t> ent_face(blk_entry[nb]);
  std::vector<int4> ent_cells(blk_entry[nb]);
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    std::vector<int32_t> list;
    for (int64_t b = lo; b < hi; ++b) {
      block_list((int)b, list);
      const int32_t e0 = blk_entry[b];
      for (size_t q = 0; q < list.size(); ++q) {
        ent_face[e0 + q] = list[q];
        ent_cells[e0 + q] = c4[list[q]];
      }
      for (int32_t c = blk_cell[b]; c < blk_cell[b + 1]; ++c) {
        int k = 0;
        for (int64_t t = icf_ptr[c]; t < icf_ptr[c + 1]; ++t) {
          const int32_t f = icf[t];
          const size_t pos = std::lower_bound(list.begin(), list.end(), f) - list.begin();
          uint16_t s16 = (uint16_t)pos;
          if (c4[f].y == c) s16 |= 0x8000u;  // sigma = -1 on c1
          slots[(size_t)c * UMAXDEG + k++] = s16;
        }
      }
    }
  });

  fl_mesh *m = new (std::nothrow) fl_mesh();
  if (!m) return fail(FL_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return fail(FL_ECUDA, "no CUDA device");
  }
  m->kind = 1;
  m->C = C;
  m->F = F;
  m->n_owned = local ? n_owned : C;
  m->n_interior = local ? n_interior : C;
  if (const fl_status sst = status_alloc(m); sst != FL_OK) {
    delete m;
    return sst;
  }
  m->renumbered = renum;
  m->cell_perm = cell_new;
  m->face_perm = face_new;
  m->face_flip.assign(F, 0);
  UnstructDev &u = m->u;
  u.n_blocks = nb;
  u.nb_interior = nb_interior;
  u.max_block_entries = max_entries;
  u.max_entries_interior = max_int;
  u.max_entries_rim = max_rim;
  u.n_entries = (int64_t)ent_face.size();
  std::vector<float> area_f(area_i.begin(), area_i.end()), ivol_f(ivol_i.begin(), ivol_i.end());
  fl_status st = FL_OK;
  if (st == FL_OK) st = upload(blk_cell, &u.blk_cell);
  if (st == FL_OK) st = upload(blk_entry, &u.blk_entry);
  if (st == FL_OK) st = upload(ent_face, &u.ent_face);
  if (st == FL_OK) st = upload(ent_cells, &u.ent_cells);
  if (st == FL_OK) st = upload(slots, &u.cell_slots);
  if (st == FL_OK) st = upload(c4, &u.face_c4);
  if (st == FL_OK) st = upload(area_i, &u.area);
  if (st == FL_OK) st = upload(vol_i, &u.vol);
  if (st == FL_OK) st = upload(ivol_i, &u.inv_vol);
  if (st == FL_OK) st = upload(area_f, &u.area_f);
  if (st == FL_OK) st = upload(ivol_f, &u.inv_vol_f);
  if (st == FL_OK && renum) st = upload(m->cell_perm, &u.perm_cell);
  if (st == FL_OK && renum) st = upload(m->face_perm, &u.perm_face);
  if (st == FL_OK && kg > 0) {
    // the stencil in internal numbering: rows by internal face, cells renamed
    std::vector<int32_t> gc((size_t)F * 2 * kg);
    std::vector<double> gw((size_t)F * 2 * kg);
    parallel_for(F, [&](int64_t lo, int64_t hi) {
      for (int64_t f = lo; f < hi; ++f) {
        const size_t src = (size_t)f * 2 * kg, dst = (size_t)face_new[f] * 2 * kg;
        for (int q = 0; q < 2 * kg; ++q) {
          gc[dst + q] = cell_new[gcell[src + q]];
          gw[dst + q] = gcoef[src + q];
        }
      }
    });
    std::vector<float> gwf(gw.begin(), gw.end());
    u.kg = kg;
    st = upload(gc, &u.gen_cell);
    if (st == FL_OK) st = upload(gw, &u.gen_coef);
    if (st == FL_OK) st = upload(gwf, &u.gen_coef_f);
  }
  if (st != FL_OK) {
    unstruct_free(m);
    status_free(m);
    delete m;
    return st;
  }
  *out = m;
  return FL_OK;
}

// The gather lists of the adjoint, built once per mesh from the device
// records (face cells, upstream cells, general stencil).
fl_status unstruct_adjoint_prepare(const fl_mesh *mc) {
  fl_mesh *m = const_cast<fl_mesh *>(mc);
  std::lock_guard<std::mutex> lock(m->adj_mu);
  UnstructDev &u = m->u;
  if (u.adj_ready) return FL_OK;
  const int64_t C = m->C, F = m->F;
  std::vector<int4> c4(F);
  if (F > 0 && cudaMemcpy(c4.data(), u.face_c4, F * sizeof(int4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(FL_ECUDA, "face record download failed");
  std::vector<int32_t> gcell;
  std::vector<double> gcoef;
  const int kg = u.kg;
  if (kg > 0) {
    gcell.resize((size_t)F * 2 * kg);
    gcoef.resize((size_t)F * 2 * kg);
    if (cudaMemcpy(gcell.data(), u.gen_cell, gcell.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(gcoef.data(), u.gen_coef, gcoef.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(FL_ECUDA, "stencil download failed");
  }
  // cell -> faces
  std::vector<int32_t> cf_ptr(C + 1, 0), cf(2 * F);
  for (int64_t f = 0; f < F; ++f) {
    cf_ptr[c4[f].x + 1]++;
    cf_ptr[c4[f].y + 1]++;
  }
  for (int64_t c = 0; c < C; ++c) cf_ptr[c + 1] += cf_ptr[c];
  {
    std::vector<int32_t> fill(cf_ptr.begin(), cf_ptr.end() - 1);
    for (int64_t f = 0; f < F; ++f) {
      cf[fill[c4[f].x]++] = (int32_t)f;
      cf[fill[c4[f].y]++] = (int32_t)f;
    }
  }
  // cell -> (face, side | k << 1) entries naming it upstream
  std::vector<int32_t> inv_ptr(C + 1, 0);
  auto for_entries = [&](auto fn) {
    for (int64_t f = 0; f < F; ++f)
      for (int side = 0; side < 2; ++side) {
        if (kg > 0) {
          for (int k = 0; k < kg; ++k) {
            const size_t i = ((size_t)f * 2 + side) * kg + k;
            if (gcoef[i] != 0.0) fn(gcell[i], f, side | (k << 1));
          }
        } else {
          const unsigned up = (unsigned)(side == 0 ? c4[f].z : c4[f].w);
          if (up != 0xFFFFFFFFu) fn((int32_t)(up & ~SIGMA_BIT), f, side);
        }
      }
  };
  for_entries([&](int32_t c, int64_t, int) { inv_ptr[c + 1]++; });
  for (int64_t c = 0; c < C; ++c) inv_ptr[c + 1] += inv_ptr[c];
  std::vector<int32_t> inv_f(inv_ptr[C]);
  std::vector<uint8_t> inv_sk(inv_ptr[C]);
  {
    std::vector<int32_t> fill(inv_ptr.begin(), inv_ptr.end() - 1);
    for_entries([&](int32_t c, int64_t f, int sk) {
      inv_f[fill[c]] = (int32_t)f;
      inv_sk[fill[c]++] = (uint8_t)sk;
    });
  }
  fl_status st = upload(cf_ptr, &u.adj_cf_ptr);
  if (st == FL_OK) st = upload(cf, &u.adj_cf);
  if (st == FL_OK) st = upload(inv_ptr, &u.adj_inv_ptr);
  if (st == FL_OK && !inv_f.empty()) st = upload(inv_f, &u.adj_inv_f);
  if (st == FL_OK && !inv_sk.empty()) st = upload(inv_sk, &u.adj_inv_sk);
  if (st == FL_OK) u.adj_ready = true;
  return st;
}

namespace {
template <class T, int LIM>
cudaError_t launch_uadj(const fl_mesh *m, const UAParams<T> &p, bool pre, cudaStream_t st) {
  if (p.C <= p.c0) return cudaSuccess;
  long long blocks = (p.C - p.c0 + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  const unsigned g = (unsigned)std::max<long long>(blocks, 1);
  const bool gen = m->u.kg > 0;
  if (gen && pre) k_unstruct_adjoint<T, LIM, true, true><<<g, 256, 0, st>>>(p);
  else if (gen) k_unstruct_adjoint<T, LIM, true, false><<<g, 256, 0, st>>>(p);
  else if (pre) k_unstruct_adjoint<T, LIM, false, true><<<g, 256, 0, st>>>(p);
  else k_unstruct_adjoint<T, LIM, false, false><<<g, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <class T>
cudaError_t run_uadj(const fl_mesh *m, int lim, const AdjArgs &s, cudaStream_t st) {
  UAParams<T> p;
  p.x = static_cast<const T *>(s.x);
  p.mu = static_cast<const T *>(s.mu);
  p.v1 = static_cast<const T *>(s.v1);
  p.v2 = static_cast<const T *>(s.v2);
  p.out = static_cast<T *>(s.out);
  const bool pre = s.cu != nullptr;
  p.u = static_cast<const T *>(pre ? s.cu : s.u);
  if (sizeof(T) == 8) {
    p.area = reinterpret_cast<const T *>(m->u.area);
    p.inv_vol = reinterpret_cast<const T *>(m->u.inv_vol);
    p.gen_coef = reinterpret_cast<const T *>(m->u.gen_coef);
  } else {
    p.area = reinterpret_cast<const T *>(m->u.area_f);
    p.inv_vol = reinterpret_cast<const T *>(m->u.inv_vol_f);
    p.gen_coef = reinterpret_cast<const T *>(m->u.gen_coef_f);
  }
  p.c4 = m->u.face_c4;
  p.gen_cell = m->u.gen_cell;
  p.kg = m->u.kg;
  p.cf_ptr = m->u.adj_cf_ptr;
  p.cf = m->u.adj_cf;
  p.inv_ptr = m->u.adj_inv_ptr;
  p.inv_f = m->u.adj_inv_f;
  p.inv_sk = m->u.adj_inv_sk;
  p.e1 = (T)s.e1;
  p.e2 = (T)s.e2;
  p.b = (T)s.b;
  p.bdt = (T)(s.cu_dt ? s.b : s.b * s.dt);
  p.bare = s.bare;
  // every owned cell (all cells of a whole mesh), or the range asked for
  p.c0 = s.chi >= 0 ? s.clo : 0;
  p.C = s.chi >= 0 ? s.chi : m->n_owned;
  switch (lim) {
    case LIM_UPWIND: return launch_uadj<T, LIM_UPWIND>(m, p, pre, st);
    case LIM_CENTRAL: return launch_uadj<T, LIM_CENTRAL>(m, p, pre, st);
    case LIM_MINMOD: return launch_uadj<T, LIM_MINMOD>(m, p, pre, st);
    case LIM_VANLEER: return launch_uadj<T, LIM_VANLEER>(m, p, pre, st);
    case LIM_SUPERBEE: return launch_uadj<T, LIM_SUPERBEE>(m, p, pre, st);
    case LIM_SMART: return launch_uadj<T, LIM_SMART>(m, p, pre, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t unstruct_adjoint(const fl_mesh *m, int lim, fl_dtype dt, const AdjArgs &s,
                             cudaStream_t st) {
  if (m->C == 0) return cudaSuccess;
  return dt == FL_F64 ? run_uadj<double>(m, lim, s, st) : run_uadj<float>(m, lim, s, st);
}

cudaError_t unstruct_scale_area(const fl_mesh *m, fl_dtype dt, const void *u, void *w, double fac,
                                cudaStream_t st) {
  if (m->F == 0) return cudaSuccess;
  long long blocks = (m->F + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  if (dt == FL_F64)
    k_scale_area_t<double><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const double *>(u), m->u.area, static_cast<double *>(w), m->F, fac);
  else
    k_scale_area_t<float><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const float *>(u), m->u.area_f, static_cast<float *>(w), m->F, (float)fac);
  return cudaGetLastError();
}

void unstruct_free(fl_mesh *m) {
  UnstructDev &u = m->u;
  void *ptrs[] = {u.blk_cell,   u.blk_entry,  u.ent_face,    u.ent_cells, u.cell_slots,
                  u.face_c4,    u.area,       u.vol,         u.inv_vol,   u.area_f,
                  u.inv_vol_f,  u.gen_cell,   u.gen_coef,    u.gen_coef_f, u.adj_cf_ptr,
                  u.adj_cf,     u.adj_inv_ptr, u.adj_inv_f,  u.adj_inv_sk, u.perm_cell,
                  u.perm_face};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  u = UnstructDev();
}

cudaError_t unstruct_stage(const fl_mesh *m, int lim, fl_dtype dt, const StageArgs &s,
                           cudaStream_t st) {
  return dt == FL_F64 ? run_ustage<double>(m, lim, s, st) : run_ustage<float>(m, lim, s, st);
}

fl_status unstruct_apply(const fl_mesh *m, int lim, fl_dtype dt, const void *theta, const void *u,
                         void *rhs, void *thf, cudaStream_t st) {
  StageArgs s;
  s.x = theta;
  s.thn = theta;
  s.y = rhs;
  s.thf = thf;
  s.u = u;
  s.seed = 2;
  cudaError_t e = unstruct_stage(m, lim, dt, s, st);
  if (e != cudaSuccess) return cuda_fail(e, "unstructured apply kernel");
  return FL_OK;
}

fl_status unstruct_step(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                        int64_t nsteps, void *theta, const void *u, void *ws, cudaStream_t st,
                        const double *gfac, void *W) {
  const size_t es = dsize(dt);
  char *wsb = static_cast<char *>(ws);
  void *A = wsb;
  void *B = wsb + align256((size_t)m->C * es);
  StageArgs s;
  s.u = u;
  s.dt = dtime;
  cudaError_t e = cudaSuccess;
  // FP64: w_f = dt A_f u_f once per call (dt > 0 keeps every sign)
  if (W != nullptr && dt == FL_F64 && dtime > 0 && m->F > 0) {
    long long blocks = (m->F + 255) / 256;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    k_scale_area<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const double *>(u), m->u.area,
                                                   static_cast<double *>(W), m->F, dtime);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "velocity pre-scaling");
    s.w = W;
  }
  if (rk == 1) {
    void *cur = theta, *nxt = A;
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
      s.x = cur; s.thn = cur; s.y = nxt; s.seed = 0; s.b = 1.0;
      s.g = gfac ? gfac[n] : 1.0;
      e = unstruct_stage(m, lim, dt, s, st);
      void *t = cur;
      cur = nxt;
      nxt = t;
    }
    if (e == cudaSuccess && cur != theta)
      e = cudaMemcpyAsync(theta, cur, m->C * es, cudaMemcpyDeviceToDevice, st);
  } else {
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
      s.x = theta; s.thn = theta; s.y = A; s.seed = 0; s.a = 0.0; s.b = 1.0;
      s.g = gfac ? gfac[3 * n] : 1.0;
      if ((e = unstruct_stage(m, lim, dt, s, st)) != cudaSuccess) break;
      s.x = A; s.thn = theta; s.y = B; s.seed = 1; s.a = 0.75; s.b = 0.25;
      s.g = gfac ? gfac[3 * n + 1] : 1.0;
      if ((e = unstruct_stage(m, lim, dt, s, st)) != cudaSuccess) break;
      s.x = B; s.thn = theta; s.y = theta; s.seed = 1; s.a = 1.0 / 3.0; s.b = 2.0 / 3.0;
      s.g = gfac ? gfac[3 * n + 2] : 1.0;
      e = unstruct_stage(m, lim, dt, s, st);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "unstructured stage kernel");
  return FL_OK;
}

cudaError_t unstruct_selection(const fl_mesh *m, fl_dtype dt, const void *u, int32_t *sel,
                               cudaStream_t st) {
  const long long nf = m->F;
  const int threads = 256;
  long long blocks = (nf + threads - 1) / threads;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  if (dt == FL_F64)
    k_unstruct_selection<double><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const double *>(u), m->u.face_c4, reinterpret_cast<int4 *>(sel), nf);
  else
    k_unstruct_selection<float><<<(unsigned)blocks, threads, 0, st>>>(
        static_cast<const float *>(u), m->u.face_c4, reinterpret_cast<int4 *>(sel), nf);
  return cudaGetLastError();
}

const double *unstruct_volumes(const fl_mesh *m) { return m->u.vol; }

}  // namespace fl
