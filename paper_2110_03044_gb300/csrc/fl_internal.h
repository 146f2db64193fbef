// fl_internal.h -- host-side definitions shared by the library's translation
// units (mesh object, error reporting, launch helpers).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
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

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline size_t dsize(fl_dtype t) { return t == FL_F64 ? 8 : 4; }
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ----------------------------------------------------------- unstructured
// Device data of a face-based mesh in the library's internal numbering.
// Cells are grouped in blocks of up to UBLOCK cells; every block owns the
// list of faces touching its cells (faces on a block boundary appear in
// both neighbouring blocks and are evaluated by both).
struct UnstructDev {
  int n_blocks = 0;
  int max_block_faces = 0;
  // per block: [cell_begin, cell_end) and [face_begin, face_end) into the
  // block face list
  int32_t *blk_cell = nullptr;   // [n_blocks + 1]
  int32_t *blk_face = nullptr;   // [n_blocks + 1]
  // block face list entries (structure of arrays)
  int32_t *bf_face = nullptr;    // internal face id (u_f index)
  int4 *bf_cells = nullptr;      // (c0, c1, up0, up1): up0 is the upstream cell when
                                 // the flow goes c0 -> c1, up1 when it goes c1 -> c0
  // per cell: local slots (index into the block's face list) of its faces,
  // with sigma in bit 15 (set when the cell is c1 of that face)
  uint16_t *cell_slots = nullptr;  // [n_cells][6]
  int32_t *face_c4 = nullptr;      // [n_faces][4] (c0, c1, up0, up1) global
  double *inv_vol = nullptr;       // [n_cells] A-free factor 1/V_c
  double *area = nullptr;          // [n_faces]
  float *inv_vol_f = nullptr;
  float *area_f = nullptr;
};

}  // namespace fl

struct fl_mesh {
  int kind = 0;  // 0 structured, 1 unstructured
  int device = 0;
  int64_t C = 0, F = 0;
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
};
