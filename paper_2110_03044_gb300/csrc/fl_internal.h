// fl_internal.h -- host-side definitions shared by the library's translation
// units (mesh object, error reporting, launch helpers).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fl.h"

namespace fl {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
fl_status fail(fl_status st, const char *fmt, ...);
fl_status cuda_fail(cudaError_t e, const char *what);

#define FL_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return ::fl::cuda_fail(e_, #expr); \
  } while (0)

#define FL_LAUNCH_CHECK(what)                               \
  do {                                                      \
    cudaError_t e_ = cudaGetLastError();                    \
    if (e_ != cudaSuccess) return ::fl::cuda_fail(e_, what); \
  } while (0)

// ------------------------------------------------------------ launch shape
// CTAs of `kernel` (with `threads` threads and `smem` dynamic bytes) that fit
// on the current device at once: occupancy per SM x SMs, cached per kernel.
int resident_ctas(const void *kernel, int threads, size_t smem);

// z-chunk length for a kernel that streams `cols` tile columns through nz
// planes, one CTA per (column, chunk): the chunk minimising
//   ceil(CTAs / resident) x (planes per chunk + prologue)
// i.e. whole waves of co-resident CTAs, each paying its z-prologue (the
// planes it loads before its first output plane) once.
int pick_zchunk(long long cols, int nz, long long resident, int prologue);

// Identity of the CUDA context current on the calling thread (the driver's
// cuCtxGetId); false when there is none or the driver lacks the call.  A
// device reset or a new primary context gives a new identity, so per-context
// state (function attributes, symbol addresses) is cached under it.
bool current_context_id(unsigned long long *id);

// Raise `kernel`'s dynamic shared-memory limit to `bytes` in the current
// context.  The attribute belongs to the context, so the call is made once
// per (kernel, context) and remembered under a lock: a process driving
// several GPUs, or one whose device was reset, sets it in every context.
cudaError_t set_smem_limit(const void *kernel, int bytes);

// The mesh status word (fl_mesh::status) lives in mapped, page-locked host
// memory: a kernel records a device-side error there with a plain store,
// and the next call on the mesh reads it on the host without synchronising.
fl_status status_alloc(fl_mesh *m);
void status_free(fl_mesh *m);

#ifdef __CUDACC__
__device__ __forceinline__ void record_status(int *status, int code) {
  *reinterpret_cast<volatile int *>(status) = code;
  __threadfence_system();
}
#endif

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline size_t dsize(fl_dtype t) { return t == FL_F64 ? 8 : 4; }
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// The weight a of an RK blend y = a thn + b (x + dt R(x)) as the kernels
// use it in precision T.  When the weights sum to 1, a = 1 - b is computed
// in T (exact: b lies in [1/2, 1] or a is 0.75 / 0), so that a + b == 1
// exactly and the blend moves no mass.  With a = RN(1/3) and b = RN(2/3),
// SSP-RK3's third stage would scale the total by 1 - 2^-54 in FP64 and by
// 1 + 2^-25 in FP32 every step.
template <class T>
inline T blend_a(double a, double b) {
  return (a + b == 1.0) ? T(1) - (T)b : (T)a;
}

// ----------------------------------------------------------- unstructured
// Device data of a face-based mesh in the library's internal numbering.
// Cells are grouped in blocks (compact patches of at most UBLOCK cells);
// every block owns the list of faces touching its cells.  A face with both
// cells in one block appears once in that block's list; a face on a block
// boundary appears in both neighbouring lists and is evaluated by both.
constexpr int UBLOCK = 512;
constexpr int UMAXDEG = 8;  // faces per cell (slot table width)

struct UnstructDev {
  int n_blocks = 0;
  int nb_interior = 0;  // local meshes: blocks [0, nb_interior) hold the interior cells
  int max_block_entries = 0;
  // the same over the interior blocks and over the rim blocks of a local
  // mesh: a launch over one range sizes its shared memory by that range
  int max_entries_interior = 0, max_entries_rim = 0;
  int64_t n_entries = 0;
  int32_t *blk_cell = nullptr;   // [n_blocks + 1] cell range of each block
  int32_t *blk_entry = nullptr;  // [n_blocks + 1] entry range of each block
  int32_t *ent_face = nullptr;   // [n_entries] internal face id
  int4 *ent_cells = nullptr;     // [n_entries] (c0, c1, up0, up1); bit 31 of
                                 // up0/up1 set when d_U = -(theta_C - theta_U)
  uint16_t *cell_slots = nullptr;  // [n_cells][UMAXDEG] entry slot within the
                                   // block, bit 15 set when the cell is c1;
                                   // 0xFFFF = unused
  int4 *face_c4 = nullptr;       // [n_faces] same record per face
  double *area = nullptr;        // [n_faces]
  double *vol = nullptr;         // [n_cells]
  double *inv_vol = nullptr;     // [n_cells]
  float *area_f = nullptr;
  float *inv_vol_f = nullptr;
  // general polyhedra (a cell face with no single opposite face): per face
  // and side (0: C = c0, 1: C = c1) kg pairs (cell, coefficient) with
  // s d_U = sum_k coef_k (theta_{cell_k} - theta_C); padding has coef 0
  int kg = 0;
  int32_t *gen_cell = nullptr;   // [n_faces][2][kg]
  double *gen_coef = nullptr;    // [n_faces][2][kg]
  float *gen_coef_f = nullptr;
  // adjoint gather lists, built on the first adjoint call: cell -> its
  // faces, and cell -> the (face, side | k << 1) upstream-stencil entries
  // that name it (hexahedra: k = 0, the single upstream cell)
  bool adj_ready = false;
  int32_t *adj_cf_ptr = nullptr;   // [n_cells + 1]
  int32_t *adj_cf = nullptr;       // [2 n_faces]
  int32_t *adj_inv_ptr = nullptr;  // [n_cells + 1]
  int32_t *adj_inv_f = nullptr;
  uint8_t *adj_inv_sk = nullptr;
  // renumbered meshes: internal index of every user cell / user face, for
  // the field order conversions (fl_mesh_to_internal / fl_mesh_to_user)
  int32_t *perm_cell = nullptr;  // [n_cells]
  int32_t *perm_face = nullptr;  // [n_faces]
};

}  // namespace fl

struct fl_mesh {
  int kind = 0;  // 0 structured, 1 unstructured
  int device = 0;
  // status word: device address for the kernels (bounded waits record
  // timeouts there) and host address of the same mapped host memory
  int *status = nullptr;
  int *status_host = nullptr;
  int64_t C = 0, F = 0;
  // face-based local meshes of a partition (fl_mesh_create_local): cells
  // [0, n_interior) and [n_interior, n_owned) are updated, the rest are halo
  // cells that no kernel writes; other meshes have n_interior = n_owned = C
  int64_t n_owned = 0, n_interior = 0;
  // structured
  int nx = 1, ny = 1, nz = 1;
  double hx = 1, hy = 1, hz = 1;
  int act[3] = {0, 0, 0};
  int64_t u_off[3] = {0, 0, 0};
  // unstructured (internal numbering); permutations on the host
  std::vector<int32_t> cell_perm, face_perm;
  std::vector<uint8_t> face_flip;
  bool renumbered = false;
  fl::UnstructDev u;
  std::mutex adj_mu;  // guards the lazy build of the adjoint lists
};
