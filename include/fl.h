/*
 * fl.h -- C ABI of the GB300 flux-limited convection library.
 *
 * The library evaluates the flux-limited convective operator of Valle et al.,
 * "On the implementation of flux limiters in algebraic frameworks", and the
 * explicit time step it drives, with hand-written sm_103a CUDA kernels.
 *
 * Operation (per face f with cells (c0, c1), unit normal n_f from c0 to c1,
 * normal velocity u_f, area A_f; per cell c with volume V_c):
 *   s_f     = u_f > 0 ? +1 : -1                        eq. (sign), Table 1 signxty
 *   C, D    = upwind / downwind cell of f (C = c0 when s_f = +1)
 *   d_u     = theta_D - theta_C                         eq. (Delta_face)
 *   d_U     = theta_C - theta_U, U the upstream cell behind C
 *             (eq. (Delta_Upwind) with the orientation correction Q)
 *   r_f     = d_U / d_u                                 eq. (gradientRatio), (rf)
 *   theta_f = theta_C + Psi(r_f) d_u / 2,  theta_f = theta_C when d_u == 0
 *                                                       eq. (FL-UP) == (FL-CD)
 *   R_c     = -(1/V_c) sum_{f in dc} sigma_cf u_f A_f theta_f,
 *             sigma = +1 when c = c0, -1 when c = c1    Algorithm 4 (M U theta_f)
 *   Euler:   theta^{n+1} = theta^n + dt R(theta^n)      Algorithm 4
 *   SSP-RK3: th1 = thn + dt R(thn); th2 = 3/4 thn + 1/4 (th1 + dt R(th1));
 *            th^{n+1} = 1/3 thn + 2/3 (th2 + dt R(th2))
 *
 * Conventions common to every call:
 *   - Field buffers (theta, u_f, rhs, lambda, workspace) are DEVICE pointers
 *     owned by the caller; the library never frees or retains them.
 *   - dtype selects the element type of every field buffer of the call:
 *     FL_F64 = double, FL_F32 = float.
 *   - Structured meshes: cell c = i + nx*(j + ny*k).  Faces exist only along
 *     axes of extent > 1; for each such axis (x, y, z order) u_f holds one
 *     block of n_cells values, the face of cell c in that block lying between
 *     c and its +1 neighbour along the axis (periodic).  n_faces = n_cells *
 *     (number of axes of extent > 1).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Compute calls are asynchronous on that stream; argument errors are
 *     returned synchronously before anything is enqueued.
 *   - Every call returns fl_status; fl_last_error() gives a thread-local
 *     message for the last failure on the calling thread.
 *   - Device-side errors (a bounded wait inside a kernel that gave up) are
 *     latched in a status word owned by the mesh, in mapped host memory.
 *     The next call on that mesh that finds one set returns it (and clears
 *     it) before running anything; fl_mesh_status synchronises a stream
 *     first and then does the same.
 *   - No compute call allocates device memory; scratch comes from the caller
 *     (fl_workspace_size / fl_adjoint_workspace_size).
 */
#ifndef FL_H_
#define FL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FL_OK = 0,
  FL_EINVAL = 1,        /* bad argument (NULL pointer, size, enum, mesh data) */
  FL_ENOMEM = 2,        /* host or device allocation failed (mesh/batch create only) */
  FL_ECUDA = 3,         /* a CUDA runtime call or a launch failed */
  FL_EUNSUPPORTED = 4,  /* valid input the library does not handle */
  FL_ENONFINITE = 5,    /* a reduction met NaN or Inf */
  FL_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  FL_EINDEX = 7         /* a cell index in the connectivity is outside [0, n_cells) */
} fl_status;

/* Limiter functions Psi(r) (Sweby's form; the paper's F(r) = (Psi - 1)/2). */
typedef enum {
  FL_UPWIND = 0,   /* Psi = 0: first-order upwind                      */
  FL_CENTRAL = 1,  /* Psi = 1: central (symmetric) reconstruction      */
  FL_MINMOD = 2,   /* max(0, min(1, r))                                */
  FL_VANLEER = 3,  /* (r + |r|) / (1 + |r|)                            */
  FL_SUPERBEE = 4, /* max(0, min(1, 2r), min(r, 2)); Table 1 superbeexty */
  FL_SMART = 5     /* max(0, min(2r, 1/4 + 3/4 r, 4))                  */
} fl_limiter;

typedef enum { FL_F32 = 0, FL_F64 = 1 } fl_dtype;

/* flags of fl_mesh_create */
#define FL_RENUMBER 1u /* reorder cells/faces internally for locality */

typedef struct fl_mesh fl_mesh;
typedef struct fl_batch fl_batch;

/* Thread-local message describing the last failure on this thread. */
const char *fl_last_error(void);

/* Library version string. */
const char *fl_version(void);

/*
 * Structured periodic box nx x ny x nz with spacings hx, hy, hz (the
 * Cartesian grid on which the method collapses to Sweby's 1D scheme,
 * Section 3.1 / Section 6).  Use ny = nz = 1 for 1D, nz = 1 for 2D.
 * periodic_mask must have the bit of every axis of extent > 1 set
 * (bit 0 = x, 1 = y, 2 = z); non-periodic boundaries return FL_EUNSUPPORTED.
 * Sizes must be >= 1 with nx*ny*nz < 2^31; spacings > 0.
 * The mesh is bound to the current CUDA device; *out owns host memory only.
 */
fl_status fl_mesh_create_structured(int nx, int ny, int nz, double hx, double hy, double hz,
                                    unsigned periodic_mask, fl_mesh **out);

/*
 * General face-based mesh (Section 2: the directed cell-to-face incidence
 * E_{C->F} given row by row as face_cells[f] = (c0, c1), plus the normal
 * matrix N_F as face_normals[f] = n_f, face areas and cell volumes).
 * All input arrays are HOST arrays, copied; the caller keeps ownership.
 *   face_cells   int32 [n_faces][2], 0 <= c < n_cells, c0 != c1
 *   face_normals double [n_faces][3], unit normal pointing c0 -> c1
 *   face_areas   double [n_faces] > 0
 *   cell_volumes double [n_cells] > 0
 * Supported meshes: cells of at most 8 faces.  The upstream difference of
 * a face f with upwind cell C is
 *   - theta_C - theta_U across the face of C opposite f, where every face
 *     of C has exactly one other face j with n_f . n_j = -+1 and the rest
 *     are orthogonal (hexahedra in any numbering and orientation);
 *   - otherwise (tetrahedra, prisms, mixed meshes) the weighted sum of eq.
 *     (Delta_Upwind), s sum_j (n_f . n_j)(theta_{j,c1} - theta_{j,c0}) over
 *     the other faces j of C, without distance weights (uniform spacing;
 *     fl_mesh_create_weighted adds Algorithm 3's distance weights).
 * Cells with more than 8 faces, and sizes of 2^31 - 1 or more, return
 * FL_EUNSUPPORTED.  A cell index outside [0, n_cells) returns FL_EINDEX.
 * Faces listed twice, c0 == c1, non-unit normals and non-positive areas or
 * volumes return FL_EINVAL.
 * With FL_RENUMBER the library reorders cells and faces into compact blocks
 * for locality.  Compute calls then take and return fields in that INTERNAL
 * order (so that a step pays nothing for the user's numbering); callers
 * holding fields in their own (user) order convert them once, before and
 * after a rollout, with fl_mesh_to_internal / fl_mesh_to_user.  Without
 * FL_RENUMBER the two orders coincide.
 */
fl_status fl_mesh_create(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                         const double *face_normals, const double *face_areas,
                         const double *cell_volumes, unsigned flags, fl_mesh **out);

/*
 * fl_mesh_create for a non-uniform mesh: face_distances[f] (HOST, double
 * [n_faces], > 0, copied) is the distance between the centres of c0 and c1.
 * The gradient ratio then compares gradients, not differences (Algorithm 3,
 * and Algorithm 2's (d_i / d_U) on a line): every term of the upstream sum
 * is divided by the distance d_j of its face and the sum is multiplied by
 * d_f, i.e.
 *   d_U = s sum_j (n_f . n_j) (d_f / d_j) (theta_{j,c1} - theta_{j,c0}),
 * and r = d_U / d_u as before.  Such meshes run the general stencil on any
 * cell shape (hexahedra included), with the weights in its coefficients.
 * Same arguments, ownership and errors as fl_mesh_create; a non-positive or
 * non-finite distance returns FL_EINVAL.  Uniform distances give the
 * results of fl_mesh_create to rounding.
 */
fl_status fl_mesh_create_weighted(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                                  const double *face_normals, const double *face_areas,
                                  const double *cell_volumes, const double *face_distances,
                                  unsigned flags, fl_mesh **out);

/*
 * The local mesh of one part of a partitioned face-based mesh (Section 4's
 * split runs; each process owns the cells of one part and keeps copies of
 * the cells its stencils reach): cells [0, n_interior) are owned and read
 * no halo cell, cells [n_interior, n_owned) are owned and read halo cells,
 * cells [n_owned, n_cells) are halo copies of other parts' cells.  Compute
 * calls on the mesh update the owned cells only and never write a halo cell.
 * A stencil of an owned cell reaches two cells deep (the face's other cell,
 * and the upstream cell behind the upwind one), so the caller gives:
 *   - every face of every owned cell and of every halo cell adjacent to an
 *     owned cell (without FL_RENUMBER, in the relative order of the whole
 *     mesh's faces: a cell then sums its faces in the whole mesh's order
 *     and gets its bits);
 *   - the cells of those faces (the second halo ring may have cut face
 *     lists: no stencil of an owned cell is taken at them).
 * face_distances: NULL, or as in fl_mesh_create_weighted.  flags: 0 or
 * FL_RENUMBER, which reorders the interior cells among themselves and the
 * rim cells among themselves into compact blocks (the halo cells and their
 * order stay as given); fl_mesh_permutation then gives the internal order,
 * in which the compute calls take their fields (a caller can build its
 * local fields in that order directly), and the cells then sum their faces
 * in the internal face order.  Other arguments and errors as
 * fl_mesh_create; FL_EINVAL unless 0 <= n_interior <= n_owned <= n_cells.
 * Multi-stage calls (fl_step_rk ...) on a local mesh run with the halo as it
 * stands; a decomposed run calls the stage entry points and refreshes the
 * halo before each.  fl_reduce_mass sums the owned cells.
 */
fl_status fl_mesh_create_local(int64_t n_cells, int64_t n_owned, int64_t n_interior,
                               int64_t n_faces, const int32_t *face_cells,
                               const double *face_normals, const double *face_areas,
                               const double *cell_volumes, const double *face_distances,
                               unsigned flags, fl_mesh **out);

/* n_owned and n_interior of a mesh (both n_cells for a whole mesh). */
fl_status fl_mesh_local_info(const fl_mesh *mesh, int64_t *n_owned, int64_t *n_interior);

/*
 * Halo gather of a partitioned run: dst[i] = src[index[i]] for i < n, the
 * values one part sends to a neighbour part (src: a cell field [n_cells] of
 * the mesh, device; index: int32 [n], device; dst: [n] device, not
 * overlapping src).  An index outside [0, n_cells) records FL_EINDEX in the
 * mesh's status word (returned by the next call) and leaves its dst entry
 * as it was.  One kernel launch.
 */
fl_status fl_halo_pack(const fl_mesh *mesh, fl_dtype dtype, const void *src,
                       const int32_t *index, int64_t n, void *dst, void *stream);

/*
 * The receiving side of fl_halo_pack: dst[index[i]] = src[i] for i < n (src:
 * [n] device; index: int32 [n] device, distinct entries; dst: a cell field
 * [n_cells] of the mesh, device, not overlapping src): the received halo
 * values of a decomposition whose ghost cells are not one slice (the rows
 * of a pencil).  An index outside [0, n_cells) records FL_EINDEX in the
 * mesh's status word and writes nothing for it.  One kernel launch.
 */
fl_status fl_halo_unpack(const fl_mesh *mesh, fl_dtype dtype, const void *src,
                         const int32_t *index, int64_t n, void *dst, void *stream);

/*
 * Internal numbering of a mesh created with FL_RENUMBER (host arrays):
 * cell_perm[user_cell] = internal cell, face_perm[user_face] = internal face,
 * face_flip[user_face] = 1 if the internal face has the opposite orientation
 * (so internal u = -user u).  Any output may be NULL.  For meshes without
 * renumbering the permutations are the identity.
 */
fl_status fl_mesh_permutation(const fl_mesh *mesh, int32_t *cell_perm, int32_t *face_perm,
                              uint8_t *face_flip);

/* Sizes of a mesh: cells, faces, kind (0 structured, 1 unstructured). */
fl_status fl_mesh_info(const fl_mesh *mesh, int64_t *n_cells, int64_t *n_faces, int *kind);

/*
 * Device-side status of the kernels run on this mesh: synchronises the
 * stream, then returns FL_ETIMEOUT (a bounded wait inside a kernel gave up)
 * if a kernel recorded it since it was last returned, and clears it.  Any
 * other call on the mesh returns a recorded error the same way, without
 * synchronising (so it sees only kernels that have finished).
 */
fl_status fl_mesh_status(const fl_mesh *mesh, void *stream);

/*
 * Field order conversion for meshes created with FL_RENUMBER (Section 2's
 * incidence E_{C->F} relabelled: the renumbering is a permutation P_c of the
 * cells and P_f of the faces, and E' = P_f E P_c^T is the same operator).
 *   kind FL_FIELD_CELL: a [n_cells] cell field (theta, rhs, lambda);
 *   kind FL_FIELD_FACE: a [n_faces] face field (u_f, theta_f).
 * fl_mesh_to_internal: dst[internal index] = src[user index];
 * fl_mesh_to_user:     dst[user index] = src[internal index];
 * with the permutation of fl_mesh_permutation (the renumbering keeps every
 * face's orientation, so no value changes sign).  src and dst: device
 * buffers of dtype elements, distinct (no aliasing: one gather or scatter
 * kernel writes dst while it reads src).  Meshes without renumbering (and
 * structured meshes) copy src to dst.  Asynchronous on `stream`.
 */
typedef enum { FL_FIELD_CELL = 0, FL_FIELD_FACE = 1 } fl_field_kind;
fl_status fl_mesh_to_internal(const fl_mesh *mesh, fl_field_kind kind, fl_dtype dtype,
                              const void *src, void *dst, void *stream);
fl_status fl_mesh_to_user(const fl_mesh *mesh, fl_field_kind kind, fl_dtype dtype,
                          const void *src, void *dst, void *stream);

fl_status fl_mesh_destroy(fl_mesh *mesh);

/*
 * Algorithm 1 plus the cell sum of Algorithm 4: evaluates
 *   rhs_c   = R(theta)_c   [n_cells]   (always)
 *   theta_f = limited face values [n_faces]   (when theta_f != NULL)
 * theta_c [n_cells], u_f [n_faces], rhs_c, theta_f: device, dtype elements.
 */
fl_status fl_conv_limited_apply(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                const void *theta_c, const void *u_f, void *rhs_c, void *theta_f,
                                void *stream);

/*
 * Upwind selection per face (eq. (sign), Delta_face, Delta_Upwind):
 * sel[f] = (s_f, C, D, U) as int32 [n_faces][4], device.  Depends on u_f
 * and the mesh only.  Cell ids in the numbering the compute calls use.
 */
fl_status fl_face_selection(const fl_mesh *mesh, fl_dtype dtype, const void *u_f, int32_t *sel,
                            void *stream);

/*
 * ---------------------------------------------------------------------------
 * The algebraic formulation (Section 3, Algorithm 1 and Algorithm 5): the
 * flux limiter built from sparse matrix-vector products (ELLPACK, 8-byte
 * values and 4-byte column indices) and pointwise kernels only, as a
 * comparison baseline for the fused stencil kernels (the paper's stencil
 * vs algebraic study, Table 2 and its performance analysis).  FP64 only.
 * ---------------------------------------------------------------------------
 */
typedef struct fl_alg fl_alg;

/*
 * Assemble, on the current device, the matrices of Algorithm 1 and of the
 * update of Algorithm 5 from an explicit face-based mesh (host arrays, the
 * layout of fl_mesh_create): E (|F| x |C|, eq. Tfc), T and -S (the two
 * precomputed operators after eq. SimplifiedDeltaUpstream, stored with the
 * sign that gives d_U = (Q T - S) theta for both flow directions), Pi
 * (eq. sCF) and M = V^-1 E^T diag(A) (|C| x |F|).  Rows keep every
 * structural entry (zero coefficients included).  Returns FL_EINDEX for
 * out-of-range cells, FL_EINVAL for self-loops, non-positive areas or
 * volumes; FL_ENOMEM when device memory runs out.  The handle owns its device
 * memory until fl_alg_destroy.
 */
fl_status fl_alg_create(int64_t n_cells, int64_t n_faces, const int32_t *face_cells,
                        const double *normals, const double *areas, const double *volumes,
                        fl_alg **out);
fl_status fl_alg_destroy(fl_alg *alg);
/* Per matrix (E, T, -S, Pi, M): structural non-zeros, ELLPACK width; total
 * device bytes of the five matrices.  Any output pointer may be NULL. */
fl_status fl_alg_info(const fl_alg *alg, int64_t *nnz /*[5]*/, int32_t *width /*[5]*/,
                      size_t *bytes);
/* Device workspace bytes of fl_alg_face_values / fl_alg_step_euler. */
fl_status fl_alg_workspace_size(const fl_alg *alg, size_t *bytes);
/*
 * Algorithm 1 as 4 SpMV + 4 pointwise launches: theta_f [n_faces] from
 * theta [n_cells] and u_f [n_faces] (device, FP64, the mesh's order).
 * u_f = 0, -0 and NaN select -1; d_u == 0 gives the upwind value.
 */
fl_status fl_alg_face_values(const fl_alg *alg, fl_limiter limiter, const void *theta,
                             const void *u_f, void *theta_f, void *workspace,
                             size_t workspace_bytes, void *stream);
/* Algorithm 5: nsteps forward-Euler steps theta <- theta + dt M U(u_f) theta_f
 * in place (Algorithm 1, then U, M and the update as 1 SpMV + 2 pointwise). */
fl_status fl_alg_step_euler(const fl_alg *alg, fl_limiter limiter, double dt, int64_t nsteps,
                            void *theta, const void *u_f, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Bytes of device workspace fl_step_rk needs (rk_order 1 or 3). */
fl_status fl_workspace_size(const fl_mesh *mesh, fl_dtype dtype, int rk_order, size_t *bytes);

/*
 * nsteps explicit steps of Algorithm 4 (rk_order 1, forward Euler) or of
 * SSP-RK3 (rk_order 3), in place on theta [n_cells] (device).  dt is the
 * physical step.  workspace: device, >= fl_workspace_size bytes, 256-byte
 * aligned; its contents are scratch.  One fused kernel launch per stage;
 * a structured 1D line of 2 .. 5120 (FP64) or 10240 (FP32) cells runs all
 * nsteps in one launch, held in shared memory (one CTA below 16 cells, a
 * cluster of 8 CTAs from 16 cells on, of 16 CTAs from 32 cells on where the
 * GPU can place such a cluster).
 */
fl_status fl_step_rk(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype, int rk_order,
                     double dt, int64_t nsteps, void *theta, const void *u_f, void *workspace,
                     size_t workspace_bytes, void *stream);

/*
 * One RK stage of fl_step_rk, for callers that sequence the stages
 * themselves (a domain decomposition that exchanges halo cells between
 * stages):
 *   y = a theta_n + b (x + dt R(x))
 * with (a, b) = (0, 1) for stage 0 (forward Euler, Algorithm 4; theta_n is
 * then unused and may be NULL) and, for rk_order 3 (SSP-RK3), (3/4, 1/4) for
 * stage 1 and (1/3, 2/3) for stage 2 (the weights sum to exactly 1 in the
 * working precision).  All buffers are device, dtype elements: theta_n, x, y
 * [n_cells], u_f, w_f [n_faces].  y must not overlap x (a stage reads the
 * neighbours of x while it writes y); y may be theta_n.  w_f: NULL, or in
 * FP64 the pre-scaled velocity of fl_velocity_prescale for the same dt,
 * with which the stage runs the arithmetic of fl_step_rk (the flux product
 * folded into the cell update) and gives its bits; without it FP64 forms
 * u_f theta_f per face.  FP32 ignores w_f.  One kernel launch; no workspace.
 */
fl_status fl_step_rk_stage(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype, int rk_order,
                           int stage, double dt, const void *theta_n, const void *x, void *y,
                           const void *u_f, const void *w_f, void *stream);

/*
 * fl_step_rk_stage over the z planes [z_begin, z_end) of a structured mesh
 * only: the cells c = i + nx (j + ny k) with z_begin <= k < z_end get the
 * bits fl_step_rk_stage gives them; y keeps its other planes.  Each updated
 * plane reads x within two planes of itself (periodic in z), so a z-slab
 * domain decomposition (Section 4's split runs) can update the planes that
 * need no ghost plane while the halo exchange is in flight, then the planes
 * next to its cuts.  Arguments as fl_step_rk_stage.  FL_EUNSUPPORTED on a
 * face-based mesh; FL_EINVAL unless 0 <= z_begin <= z_end <= nz (an empty
 * range runs nothing).  One kernel launch.
 */
fl_status fl_step_rk_stage_planes(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                  int rk_order, int stage, double dt, int z_begin, int z_end,
                                  const void *theta_n, const void *x, void *y, const void *u_f,
                                  const void *w_f, void *stream);

/*
 * fl_step_rk_stage over the rows [y_begin, y_end) of the planes [z_begin,
 * z_end) of a structured mesh only (the cells i + nx (j + ny k) with j and k
 * in range, every i): a pencil decomposition's interior and rim boxes.  Each
 * updated cell reads x within two cells of itself along each axis (periodic).
 * Arguments as fl_step_rk_stage_planes; FL_EINVAL unless 0 <= y_begin <=
 * y_end <= ny and 0 <= z_begin <= z_end <= nz (an empty box runs nothing).
 * One kernel launch.
 */
fl_status fl_step_rk_stage_box(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                               int rk_order, int stage, double dt, int y_begin, int y_end,
                               int z_begin, int z_end, const void *theta_n, const void *x, void *y,
                               const void *u_f, const void *w_f, void *stream);

/*
 * fl_step_rk_stage over the owned cells [c_begin, c_end) of a local mesh
 * (fl_mesh_create_local) only; each end is 0, n_interior or n_owned, so a
 * partitioned run can update its interior cells while the halo exchange is
 * in flight and the cells next to the halo after it.  Cells outside the
 * range keep their values in y.  FL_EUNSUPPORTED on a structured mesh;
 * FL_EINVAL for another range.  One kernel launch.
 */
fl_status fl_step_rk_stage_cells(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                 int rk_order, int stage, double dt, int64_t c_begin,
                                 int64_t c_end, const void *theta_n, const void *x, void *y,
                                 const void *u_f, const void *w_f, void *stream);

/*
 * w_f = dt (A_f / V) u_f per face (Algorithm 4's M U with the step size:
 * structured meshes take A/V = 1/h of the face's axis, face-based meshes
 * w_f = dt A_f u_f with 1/V applied per cell), the velocity fl_step_rk_stage
 * takes as w_f.  A product that underflows keeps the sign of u_f, so the
 * upwind side of every face is unchanged.  dt must be finite and > 0.
 * u_f, w_f: device, [n_faces] dtype elements.
 */
fl_status fl_velocity_prescale(const fl_mesh *mesh, fl_dtype dtype, double dt, const void *u_f,
                               void *w_f, void *stream);

/*
 * fl_step_rk for a time-modulated flow: stage s of step n advects with the
 * face velocity g[n * S + s] * u_f (S = 1 for Euler, 3 for SSP-RK3), the
 * form of the reversing deformation flow of Section 4.1 (eq. rhodonea),
 * whose velocity is a fixed field times cos(pi t / T).  g: host array of
 * nsteps * S finite factors, read before the call returns.  A negative
 * factor reverses every face's upwind side (the sign of g u_f decides, so
 * u_f = 0 still selects -1).  Same workspace, ownership and errors as
 * fl_step_rk; a non-finite factor returns FL_EINVAL before any launch.
 */
fl_status fl_step_rk_modulated(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                               int rk_order, double dt, int64_t nsteps, void *theta,
                               const void *u_f, const double *g, void *workspace,
                               size_t workspace_bytes, void *stream);

/*
 * fl_step_rk with temporal blocking, for structured meshes: one kernel launch
 * runs all three stages of an SSP-RK3 step (rk_order 3) or three forward-Euler
 * steps of Algorithm 4 (rk_order 1), so that theta^n and u_f are read from
 * device memory once per launch instead of once per stage.  The paper
 * evaluates one operator application at a time; this is the same arithmetic
 * (Algorithm 1's limited face values, Algorithm 4's update, the SSP-RK3
 * blends) with each stage's halo recomputed on chip, two cells per stage and
 * side.  Results agree with fl_step_rk to rounding: both meet the same
 * bounds against the FP64 oracle (FP64 here forms u_f theta_f per face where
 * fl_step_rk folds dt (A/V) u_f into the cell update).
 * Same arguments, ownership and workspace as fl_step_rk (the workspace holds
 * the other half of a ping-pong pair; the result is copied back into theta
 * when it lands there).  Euler steps beyond a multiple of three run stage by
 * stage.  A face-based mesh returns FL_EUNSUPPORTED before any launch.
 */
fl_status fl_step_rk_blocked(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                             int rk_order, double dt, int64_t nsteps, void *theta,
                             const void *u_f, void *workspace, size_t workspace_bytes,
                             void *stream);

/*
 * fl_step_rk without a workspace argument, for callers that may not allocate
 * device memory at all (plugin hosts that own the whole device memory pool,
 * real-time loops that cannot pay for an allocation's device-wide
 * synchronisation, deployments whose memory is fixed at start-up).  The paper
 * has no counterpart: this is a deployment convenience of the library.
 * Same arguments and results as fl_step_rk; the stage buffers come from a
 * fixed area inside the library image of FL_NOALLOC_SCRATCH_BYTES per GPU,
 * held by every GPU that loads the library until the process exits.  Meshes
 * whose RK stage buffers (|C| values for Euler, two blocks of |C| for SSP-RK3,
 * each rounded up to 256 bytes) exceed that return FL_EINVAL and nothing
 * runs.  (fl_step_rk's FP64 workspace also holds a pre-scaled copy of u_f;
 * this entry point runs the same stages without it.)
 * The first call on each device looks up the area's device address, so make
 * it before any stream capture.  The address is remembered with the identity
 * of the CUDA context it was taken in; after a device reset (a new context)
 * the next call looks it up again.  All calls share the area: calls whose GPU
 * work overlaps in time race and must be ordered by the caller.  The call
 * allocates nothing (no cudaMalloc, no library allocator).
 */
#define FL_NOALLOC_SCRATCH_BYTES (32u << 20)
fl_status fl_step_rk_noalloc(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                             int rk_order, double dt, int64_t nsteps, void *theta,
                             const void *u_f, void *stream);

/*
 * Transpose of the Jacobian of R at theta_c applied to lambda_rhs:
 *   lambda_theta = (dR/dtheta)^T lambda_rhs     [n_cells] device.
 * The limiter derivative is taken on the branch selected by strict ordered
 * tests at theta_c (ties to the lower branch); d_u == 0 keeps theta_C.
 */
fl_status fl_conv_limited_adjoint(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                  const void *theta_c, const void *u_f, const void *lambda_rhs,
                                  void *lambda_theta, void *stream);

/*
 * Reverse mode of one RK stage of fl_step_rk_stage, for callers that run the
 * reverse sweep themselves (a domain decomposition that exchanges the
 * adjoint's halo between stages).  Stage s maps
 *   y_s = a_s theta_n + b_s (x_s + dt R(x_s))
 * ((a_s, b_s) as in fl_step_rk_stage).  Given mu = dJ/dy_s it writes
 *   stage s > 0:  out = b_s (mu + dt R'(x_s)^T mu)              (= dJ/dx_s)
 *   stage 0:      out = mu + dt R'(theta_n)^T mu                 (Euler), or
 *                 out = mu + dt R'(theta_n)^T mu + a_1 lam_a + a_2 lam_b
 *                 (SSP-RK3: theta_n's other uses, in the blends of stages 1
 *                 and 2, with lam_a = dJ/dy_1 and lam_b = dJ/dy_2)
 * so that one SSP-RK3 step back from lambda = dJ/dtheta^{n+1} is
 *   m2 = stage 2 (x_2, lambda);  m1 = stage 1 (x_1, m2);
 *   dJ/dtheta^n = stage 0 (theta^n, m1, lam_a = m2, lam_b = lambda).
 * The limiter derivative is taken on the branch its forward evaluation at
 * x_s takes (strict ordered tests, ties to the lower branch).  All buffers
 * device, dtype elements: x, mu, lam_a, lam_b, out [n_cells]; u_f, w_f
 * [n_faces].  lam_a, lam_b are read only in stage 0 of SSP-RK3 (else they
 * may be NULL).  out must not overlap x or mu; it may be lam_a or lam_b.
 * w_f: NULL, or the pre-scaled velocity of fl_velocity_prescale for the same
 * dt.  Reads mu within two cells and x within three cells of each output.
 * The paper has no adjoint; this is defined by the forward steps above.
 */
fl_status fl_step_rk_stage_adjoint(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                   int rk_order, int stage, double dt, const void *x,
                                   const void *mu, const void *lam_a, const void *lam_b,
                                   void *out, const void *u_f, const void *w_f, void *stream);

/*
 * fl_step_rk_stage_adjoint over the z planes [z_begin, z_end) of a
 * structured mesh only (out keeps its other planes), the reverse
 * counterpart of fl_step_rk_stage_planes: an updated plane reads mu within
 * two planes and x within three planes of itself.  Arguments as
 * fl_step_rk_stage_adjoint; FL_EUNSUPPORTED on a face-based mesh, FL_EINVAL
 * unless 0 <= z_begin <= z_end <= nz.  One kernel launch.
 */
fl_status fl_step_rk_stage_adjoint_planes(const fl_mesh *mesh, fl_limiter limiter,
                                          fl_dtype dtype, int rk_order, int stage, double dt,
                                          int z_begin, int z_end, const void *x, const void *mu,
                                          const void *lam_a, const void *lam_b, void *out,
                                          const void *u_f, const void *w_f, void *stream);

/*
 * fl_step_rk_stage_adjoint over the rows [y_begin, y_end) of the planes
 * [z_begin, z_end) of a structured mesh only: an updated cell reads mu
 * within two cells and x within three cells of itself along each axis.
 * Errors as fl_step_rk_stage_box.
 */
fl_status fl_step_rk_stage_adjoint_box(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                       int rk_order, int stage, double dt, int y_begin,
                                       int y_end, int z_begin, int z_end, const void *x,
                                       const void *mu, const void *lam_a, const void *lam_b,
                                       void *out, const void *u_f, const void *w_f, void *stream);

/*
 * fl_step_rk_stage_adjoint over the owned cells [c_begin, c_end) of a local
 * mesh only (each end 0, n_interior or n_owned): an owned cell's output
 * reads mu and x within two cells of it.  Errors as fl_step_rk_stage_cells.
 */
fl_status fl_step_rk_stage_adjoint_cells(const fl_mesh *mesh, fl_limiter limiter,
                                         fl_dtype dtype, int rk_order, int stage, double dt,
                                         int64_t c_begin, int64_t c_end, const void *x,
                                         const void *mu, const void *lam_a, const void *lam_b,
                                         void *out, const void *u_f, const void *w_f,
                                         void *stream);

/* Bytes of device workspace fl_step_rk_adjoint needs. */
fl_status fl_adjoint_workspace_size(const fl_mesh *mesh, fl_dtype dtype, int rk_order,
                                    int64_t nsteps, int64_t checkpoint_every, size_t *bytes);

/*
 * Reverse-mode sweep of nsteps steps from theta0: given lambda_T = dJ/dtheta_T
 * returns lambda_0 = dJ/dtheta_0 (all [n_cells], device).  The forward
 * rollout is checkpointed every checkpoint_every steps in the workspace and
 * each segment is recomputed (storing its stage states) before its adjoint
 * stages run in reverse order.  theta0 is not modified.
 */
fl_status fl_step_rk_adjoint(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                             int rk_order, double dt, int64_t nsteps, int64_t checkpoint_every,
                             const void *theta0, const void *u_f, const void *lambda_T,
                             void *lambda_0, void *workspace, size_t workspace_bytes,
                             void *stream);

/*
 * The two halves of fl_step_rk_adjoint, for callers that run the forward
 * rollout themselves (e.g. an autograd forward pass) and want the reverse
 * sweep without rerunning the checkpointing pass:
 *   fl_step_rk_checkpointed advances theta (in place, nsteps steps) and
 *     stores a checkpoint every checkpoint_every steps in the workspace;
 *   fl_step_rk_adjoint_from_checkpoints then runs the reverse sweep from
 *     those checkpoints (same mesh, limiter, dtype, rk_order, dt, nsteps,
 *     checkpoint_every, u_f and workspace, contents untouched in between).
 * Workspace: fl_adjoint_workspace_size bytes.
 */
fl_status fl_step_rk_checkpointed(const fl_mesh *mesh, fl_limiter limiter, fl_dtype dtype,
                                  int rk_order, double dt, int64_t nsteps,
                                  int64_t checkpoint_every, void *theta, const void *u_f,
                                  void *workspace, size_t workspace_bytes, void *stream);
fl_status fl_step_rk_adjoint_from_checkpoints(const fl_mesh *mesh, fl_limiter limiter,
                                              fl_dtype dtype, int rk_order, double dt,
                                              int64_t nsteps, int64_t checkpoint_every,
                                              const void *u_f, const void *lambda_T,
                                              void *lambda_0, void *workspace,
                                              size_t workspace_bytes, void *stream);

/*
 * Batched form: n independent structured meshes advanced together, one
 * persistent launch per stage over all instances.  meshes: host array of n
 * structured meshes (kept by reference; they must outlive the batch).
 */
fl_status fl_batch_create(int n, const fl_mesh *const *meshes, fl_batch **out);

/*
 * Workspace bytes of fl_batch_step_rk: per box its RK stage buffers (and in
 * FP64 its pre-scaled velocities); in FP32 at least the padded copy of
 * decomposition kind 2 (theta, the stage buffers and the velocities of each
 * box with nx >= 8 at (nx + 4 rounded up to 4) x (ny + 4) x (nz + 4) cells,
 * the 4 dropped along an axis of one cell), whichever is larger.
 */
fl_status fl_batch_workspace_size(const fl_batch *batch, fl_dtype dtype, int rk_order,
                                  size_t *bytes);

/*
 * nsteps steps of every instance.  theta, u_f: host arrays of n device
 * pointers; dt: host array of n step sizes.  The work items of all
 * instances (see fl_batch_tiling) form one list; every stage is one
 * persistent launch over it, replayed from a captured CUDA graph.  The batch owns one
 * parameter table and one set of work counters, so calls on one batch run in
 * call order: a call's stream first waits for the previous call's launches
 * (an event recorded on that call's stream), whichever stream that was.
 * Calls on one batch from several host threads at once are not supported.
 */
fl_status fl_batch_step_rk(fl_batch *batch, fl_limiter limiter, fl_dtype dtype, int rk_order,
                           const double *dt, int64_t nsteps, void *const *theta,
                           const void *const *u_f, void *workspace, size_t workspace_bytes,
                           void *stream);

/*
 * The work decomposition of a batch's persistent launch for (limiter, dtype,
 * rk_order): as the autotuner picked it on the first fl_batch_step_rk call
 * with these arguments (timing a few stage launches of each candidate), or
 * as fl_batch_set_tiling fixed it.
 *   kind 0: rectangles of 32 x 8 cells, one cell per thread (FP64 and FP32);
 *   kind 1: runs of 32 x cells_per_thread x warps consecutive cells of a
 *           plane in the flat order c = i + nx j, a thread's cells 32 apart
 *           (FP32 only);
 *   kind 2: runs of 128 x warps cells of a plane of a padded copy of each
 *           box (periodic ghost cells, rows padded to a multiple of 4), a
 *           thread holding 4 consecutive cells (FP32 only).  The call copies
 *           theta and u_f into the workspace's padded copies before the first
 *           step and theta back after the last; boxes with nx < 8, or whose
 *           padded copy would hold 2^31 cells or more, stay in their own
 *           layout and run kind 1's tile with one cell per thread over runs
 *           of 32 x warps;
 *   z_chunk: planes per work item.
 * fl_batch_tiling returns FL_EINVAL until a decomposition exists; any
 * output pointer may be NULL.  fl_batch_set_tiling validates the choice
 * (kind 0: cells_per_thread 1, warps 8; kind 1: FP32, cells_per_thread 1, 2
 * or 4, warps 1 .. 8; kind 2: FP32, cells_per_thread 4, warps 1 .. 8;
 * z_chunk 1 .. 255) and skips the autotuner.
 */
fl_status fl_batch_tiling(const fl_batch *batch, fl_limiter limiter, fl_dtype dtype, int rk_order,
                          int *kind, int *cells_per_thread, int *warps, int *z_chunk);
fl_status fl_batch_set_tiling(fl_batch *batch, fl_limiter limiter, fl_dtype dtype, int rk_order,
                              int kind, int cells_per_thread, int warps, int z_chunk);

fl_status fl_batch_destroy(fl_batch *batch);

/*
 * kred-style reductions (Section 3.2 generalised reduction):
 *   fl_reduce_max_abs: *out = max_i |x_i| over n elements (e.g. max |u_f|
 *                      for the CFL step size); FL_ENONFINITE if any x_i is
 *                      NaN or Inf.
 *   fl_reduce_mass:    *out = sum_c V_c theta_c (conserved quantity) for a
 *                      mesh's cells, compensated summation; FL_ENONFINITE on
 *                      NaN/Inf.
 * x / theta: device; out: HOST double.  These calls synchronise the stream.
 * workspace: device, >= fl_reduce_workspace_size() bytes.
 */
size_t fl_reduce_workspace_size(void);
fl_status fl_reduce_max_abs(fl_dtype dtype, const void *x, int64_t n, double *out,
                            void *workspace, void *stream);
fl_status fl_reduce_mass(const fl_mesh *mesh, fl_dtype dtype, const void *theta, double *out,
                         void *workspace, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FL_H_ */
