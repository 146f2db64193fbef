// fl_unstructured.cu -- placeholder until the face-based kernels land.
#include "fl_unstructured.h"

namespace fl {

fl_status unstruct_create(int64_t, int64_t, const int32_t *, const double *, const double *,
                          const double *, unsigned, fl_mesh **) {
  return fail(FL_EUNSUPPORTED, "face-based meshes not available in this build");
}
void unstruct_free(fl_mesh *) {}
fl_status unstruct_apply(const fl_mesh *, int, fl_dtype, const void *, const void *, void *, void *,
                         cudaStream_t) {
  return fail(FL_EUNSUPPORTED, "face-based meshes not available in this build");
}
fl_status unstruct_step(const fl_mesh *, int, fl_dtype, int, double, int64_t, void *, const void *,
                        void *, cudaStream_t) {
  return fail(FL_EUNSUPPORTED, "face-based meshes not available in this build");
}
cudaError_t unstruct_selection(const fl_mesh *, fl_dtype, const void *, int32_t *, cudaStream_t) {
  return cudaErrorNotSupported;
}
const double *unstruct_volumes(const fl_mesh *) { return nullptr; }

}  // namespace fl
