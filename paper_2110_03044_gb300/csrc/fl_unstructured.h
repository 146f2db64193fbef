// fl_unstructured.h -- face-based (renumbered) meshes: host build and kernels.
#pragma once

#include <cuda_runtime.h>

#include "fl_internal.h"

namespace fl {

// distances: face distances d_f of a non-uniform mesh, or null (uniform)
// n_owned / n_interior: the updated cells of a local mesh (both C for a whole mesh)
fl_status unstruct_create(int64_t C, int64_t F, const int32_t *face_cells, const double *normals,
                          const double *areas, const double *volumes, const double *distances,
                          unsigned flags, int64_t n_owned, int64_t n_interior, fl_mesh **out);
void unstruct_free(fl_mesh *m);
fl_status unstruct_apply(const fl_mesh *m, int lim, fl_dtype dt, const void *theta, const void *u,
                         void *rhs, void *thf, cudaStream_t st);
fl_status unstruct_step(const fl_mesh *m, int lim, fl_dtype dt, int rk, double dtime,
                        int64_t nsteps, void *theta, const void *u, void *ws, cudaStream_t st,
                        const double *gfac = nullptr, void *W = nullptr);
cudaError_t unstruct_selection(const fl_mesh *m, fl_dtype dt, const void *u, int32_t *sel,
                               cudaStream_t st);
const double *unstruct_volumes(const fl_mesh *m);
struct AdjArgs;
// adjoint of one stage on a face-based mesh (fl_kernels.h's AdjArgs)
fl_status unstruct_adjoint_prepare(const fl_mesh *m);
cudaError_t unstruct_adjoint(const fl_mesh *m, int lim, fl_dtype dt, const AdjArgs &s,
                             cudaStream_t st);
// w_f = fac A_f u_f (internal face order)
cudaError_t unstruct_scale_area(const fl_mesh *m, fl_dtype dt, const void *u, void *w, double fac,
                                cudaStream_t st);
struct StageArgs;
cudaError_t unstruct_stage(const fl_mesh *m, int lim, fl_dtype dt, const StageArgs &s,
                           cudaStream_t st);

}  // namespace fl
