// fl_kernels.h -- launchers implemented in the .cu files (internal).
#pragma once

#include <cuda_runtime.h>

#include "fl_internal.h"

namespace fl {

// One RK stage y = a*thn + b*(x + dt R(x)) (seed 1), y = x + dt R(x)
// (seed 0, b = 1) or y = R(x) plus optional theta_f (seed 2).
struct StageArgs {
  const void *x = nullptr;
  const void *thn = nullptr;
  void *y = nullptr;
  void *thf = nullptr;
  const void *u = nullptr;
  const void *w = nullptr;  // dt (A/V) u_f, or null (see struct_scale_faces)
  double a = 0.0, b = 1.0, dt = 0.0;
  double g = 1.0;  // velocity factor of the stage: the flow is g u_f
  void *codes = nullptr;  // FP64 pre-scaled stages: branch code per face out (or null)
  int seed = 0;
  int zlo = 0, zhi = -1;  // structured meshes: update planes [zlo, zhi) only (zhi < 0: all)
  int ylo = 0, yhi = -1;  // ... and rows [ylo, yhi) of them (yhi < 0: all)
  // face-based local meshes: update cells [clo, chi) only (chi < 0: every
  // owned cell); a stage takes 0, n_interior or n_owned as either end
  int64_t clo = 0, chi = -1;
};

cudaError_t struct_stage(const fl_mesh *m, int lim, fl_dtype dt, const StageArgs &s,
                         cudaStream_t st);
// FP32 TMA-staged variant (fl_struct_tma.cu): eligibility and launch;
// returns cudaErrorNotSupported when the tensor maps cannot be built
bool struct_tma_eligible(const fl_mesh *m, const StageArgs &s);
cudaError_t struct_stage_tma(const fl_mesh *m, int lim, const StageArgs &s, cudaStream_t st);
// w_f = (fac / h_axis) u_f over the mesh's face blocks (sign kept on underflow)
cudaError_t struct_scale_faces(const fl_mesh *m, fl_dtype dt, const void *u, void *w, double fac,
                               cudaStream_t st);
// whether struct_step uses a pre-scaled velocity buffer for this mesh / dtype
bool struct_step_prescales(const fl_mesh *m, fl_dtype dt);
// nsteps Euler / SSP-RK3 steps through struct_stage; A (and B for RK3) hold
// |C| values each; W (|F| values, or null) receives dt (A/V) u_f; gfac (host,
// nsteps x stages, or null) gives each stage's velocity factor
cudaError_t struct_step(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                        int64_t nsteps, void *theta, const void *u, void *A, void *B, void *W,
                        cudaStream_t st, const double *gfac = nullptr);
// temporally blocked steps (fl_struct_fused.cu): each launch runs one
// SSP-RK3 step (rk 3) or three Euler steps (rk 1) from theta into Y (|C|
// values) and the result returns to theta; Euler steps beyond a multiple of
// three run through struct_step with Y as its stage buffer
cudaError_t struct_step_fused(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                              int64_t nsteps, void *theta, const void *u, void *Y,
                              cudaStream_t st);
size_t struct_fused_smem_bytes(fl_dtype dt);
size_t line_resident_max_cells(fl_dtype dt);
// whether the one-CTA resident kernel runs a structured mesh's steps: a
// periodic line of 2 .. line_resident_max_cells cells (a 1 x 1 x 1 mesh has
// no faces and takes the tiled kernel, which reads no velocity there)
bool line_resident_takes(const fl_mesh *m, fl_dtype dt);
cudaError_t line_resident(const fl_mesh *m, int lim, fl_dtype dt, void *theta, const void *u,
                          int64_t nsteps, int rk, double dtime, cudaStream_t st);
cudaError_t struct_selection(const fl_mesh *m, fl_dtype dt, const void *u, int32_t *sel,
                             cudaStream_t st);

// Adjoint of one stage: out = e1 v1 + e2 v2 + b mu + b dt R'(x)^T mu, or
// out = R'(x)^T mu when bare.  v1, v2 may be null; out may alias v1 / v2.
struct AdjArgs {
  const void *x = nullptr;
  const void *mu = nullptr;
  const void *v1 = nullptr;
  const void *v2 = nullptr;
  void *out = nullptr;
  const void *u = nullptr;
  const void *cu = nullptr;  // u_f pre-multiplied by A/V of its axis, or null
  int cu_dt = 0;             // cu also carries the factor dt (then b replaces b dt)
  const void *codes = nullptr;  // branch codes of the forward stage at x, or null
  double e1 = 0.0, e2 = 0.0, b = 1.0, dt = 0.0;
  int bare = 0;
  int zlo = 0, zhi = -1;  // structured meshes: update planes [zlo, zhi) only (zhi < 0: all)
  int ylo = 0, yhi = -1;  // ... and rows [ylo, yhi) of them (yhi < 0: all)
  // face-based local meshes: update cells [clo, chi) only (chi < 0: every
  // owned cell); a stage takes 0, n_interior or n_owned as either end
  int64_t clo = 0, chi = -1;
};

cudaError_t struct_adjoint(const fl_mesh *m, int lim, fl_dtype dt, const AdjArgs &s,
                           cudaStream_t st);
size_t adjoint_ws_bytes(const fl_mesh *m, fl_dtype dt, int rk, int64_t nsteps, int64_t every);

// reductions (fl_reduce.cu)
size_t reduce_ws_bytes();
cudaError_t reduce_max_abs(fl_dtype dt, const void *x, int64_t n, void *ws, cudaStream_t st,
                           double *out, int *nonfinite);
cudaError_t reduce_mass(fl_dtype dt, const void *theta, const double *vol, double vconst,
                        int64_t n, void *ws, cudaStream_t st, double *out, int *nonfinite);

}  // namespace fl
