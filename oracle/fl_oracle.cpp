// fl_oracle.cpp -- plain, slow, FP64 CPU reference of the flux-limited
// convective operator and the explicit time step it drives.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library (the CUDA path) may call,
// link or load this file; only the test suite, the smoke check and the CPU
// baseline leg of the benchmark use it.  It shares no code, header, table or
// constant with the CUDA path.
//
// What it computes (Valle et al., "On the implementation of flux limiters in
// algebraic frameworks"):
//   * Section 3, eq. (FL-UP) / (FL-CD): limited face value
//       theta_f = theta_C + Psi(r) (theta_D - theta_C) / 2
//   * eq. (gradientRatio) / (rf): r_f = Delta_U theta / Delta_u theta
//   * eq. (sign): upwind side from sign(u_f), with u_f > 0 ? +1 : -1
//     (Table 1, kernel signxty), so u_f == 0, -0 and NaN select -1
//   * eq. (Delta_face): d_u = Q E theta  = theta_D - theta_C
//   * eq. (Delta_Upwind): upstream difference accumulated over the other faces
//     j of the upstream cell C, each projected on n_f:
//       d_U = s * sum_{j in dC, j != f} (n_f . n_j) (theta_{j,c1} - theta_{j,c0})
//     The leading factor s is a sign correction: each printed form of d_U
//     agrees with Sweby's r for one flow direction only, and the
//     orientation-invariant sum times s = sign(u_f) agrees for both.  On
//     hexahedral meshes this is exactly theta_C - theta_U.  Non-uniform
//     meshes given face distances d_f take Algorithm 3's weights (Algorithm
//     2's d_i / d_U in 1D): each term is divided by d_j and the sum
//     multiplied by d_f, so r compares gradients, not differences.
//   * Algorithm 4: theta^{n+1} = theta^n + dt M U(u_f) theta_f, with M read as
//     minus the divergence: R_c = -(1/V_c) sum_f sigma_cf u_f A_f theta_f,
//     sigma = +1 when c is c0 of f and -1 when c is c1.
//   * SSP-RK3 (Shu-Osher) stages built from the same R (the paper uses forward
//     Euler; RK3 is the standard three-stage TVD scheme).
//   * Tangent-linear and adjoint (transpose) of one stage, with the limiter
//     derivative taken on the branch selected by strict ordered tests.
//
// Build: g++ -O2 -fno-fast-math -ffp-contract=off [-fopenmp] -shared -fPIC.
// FP64, round-to-nearest, no FMA contraction, fixed per-cell face order (the
// order of the cell's faces in ascending face index).
//
// Conventions: face f has cells (c0, c1) and unit normal n_f pointing c0->c1;
// u_f is the normal velocity along n_f; A_f face area; V_c cell volume.
//
// Pins (tests/test_oracle_*.py): every function here is checked against
// something other than itself -- the paper's printed 2D example, tabulated
// closed-form limiter values, dense matrix algebra of Algorithm 1 on small
// meshes, exact upwind shifts and Fourier amplification factors,
// conservation, the 3D -> 1D collapse, central differences for the
// tangent-linear model, and the adjoint dot-product identity -- and planted
// mistakes in a copy of this file must fail those pins.  Parity unpinned:
// boundedness of SMART (outside Sweby's region) and of 3D unsplit steps,
// which are reported, not asserted.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { L_UPWIND = 0, L_CENTRAL = 1, L_MINMOD = 2, L_VANLEER = 3, L_SUPERBEE = 4, L_SMART = 5 };

struct OMesh {
  int64_t C = 0, F = 0;
  std::vector<int32_t> c0, c1;        // face -> cells
  std::vector<double> nx, ny, nz;     // face normals
  std::vector<double> area;           // face areas
  std::vector<double> vol;            // cell volumes
  std::vector<int64_t> cf_ptr;        // cell -> faces (CSR), ascending face id
  std::vector<int64_t> cf_idx;
  std::vector<double> dist;           // face distances d_f (empty: uniform mesh)
};

// Algorithm 3's distance weighting (and Algorithm 2's d_i / d_U in 1D): the
// contribution of face j to the upstream gradient is divided by its
// distance d_j, and r compares that gradient with the face's own,
// (theta_D - theta_C) / d_f.  So d_U carries the factor d_f / d_j per term.
// Meshes given without distances (uniform spacing) take no weights.
inline double dist_term(const OMesh &m, double term, int64_t j) {
  return m.dist.empty() ? term : term / m.dist[j];
}
inline double dist_face(const OMesh &m, double acc, int64_t f) {
  return m.dist.empty() ? acc : acc * m.dist[f];
}

// ---------------------------------------------------------------- limiters
// Closed forms (Sweby's Psi; F(r) = (Psi - 1)/2 in the paper's notation).
//   superbee: Table 1 (superbeexty) and the expression after Algorithm 1
//   minmod, van Leer, SMART: standard r-forms of these limiters.
double psi_closed(int lim, double r) {
  switch (lim) {
    case L_UPWIND: return 0.0;
    case L_CENTRAL: return 1.0;
    case L_MINMOD: return std::fmax(0.0, std::fmin(1.0, r));
    case L_VANLEER:
      // (r + |r|) / (1 + |r|), written for r > 0 as 2 r / (1 + r) with the
      // quotient taken first so that r -> +inf gives 2 instead of inf/inf.
      if (r > 0.0) {
        if (std::isinf(r)) return 2.0;
        return 2.0 * (r / (1.0 + r));
      }
      return 0.0;
    case L_SUPERBEE:
      return std::fmax(0.0, std::fmax(std::fmin(1.0, 2.0 * r), std::fmin(r, 2.0)));
    case L_SMART:
      return std::fmax(0.0, std::fmin(std::fmin(2.0 * r, 0.25 + 0.75 * r), 4.0));
  }
  return std::nan("");
}

// Piecewise form used for derivatives: returns Psi and sets dpsi = Psi'(r).
// Branches are chosen by strict ordered tests (ties go to the lower branch).
double psi_branch(int lim, double r, double *dpsi) {
  switch (lim) {
    case L_UPWIND: *dpsi = 0.0; return 0.0;
    case L_CENTRAL: *dpsi = 0.0; return 1.0;
    case L_MINMOD:
      if (r <= 0.0) { *dpsi = 0.0; return 0.0; }
      if (r <= 1.0) { *dpsi = 1.0; return r; }
      *dpsi = 0.0; return 1.0;
    case L_VANLEER:
      if (r <= 0.0) { *dpsi = 0.0; return 0.0; }
      if (std::isinf(r)) { *dpsi = 0.0; return 2.0; }
      *dpsi = 2.0 / ((1.0 + r) * (1.0 + r));
      return 2.0 * (r / (1.0 + r));
    case L_SUPERBEE:
      if (r <= 0.0) { *dpsi = 0.0; return 0.0; }
      if (r <= 0.5) { *dpsi = 2.0; return 2.0 * r; }
      if (r <= 1.0) { *dpsi = 0.0; return 1.0; }
      if (r <= 2.0) { *dpsi = 1.0; return r; }
      *dpsi = 0.0; return 2.0;
    case L_SMART:
      if (r <= 0.0) { *dpsi = 0.0; return 0.0; }
      // r = +inf (a subnormal d_u) lies on the cap; the test below would
      // compare inf <= inf
      if (std::isinf(r)) { *dpsi = 0.0; return 4.0; }
      if (2.0 * r <= 0.25 + 0.75 * r) { *dpsi = 2.0; return 2.0 * r; }
      if (0.25 + 0.75 * r <= 4.0) { *dpsi = 0.75; return 0.25 + 0.75 * r; }
      *dpsi = 0.0; return 4.0;
  }
  *dpsi = std::nan("");
  return std::nan("");
}

// Psi'(r) of the branch the exact ratio r = dU / du (du != 0) lies on.  The
// branch is decided without the rounded quotient: with p = dU sign(du) and
// q = |du| > 0, r <= k is kd p <= kn q for k = kn / kd, and the sign of
// kd p - kn q is exact (p, q and the difference are multiples of 2^-1074,
// so the one fma or subtraction that forms it only rounds a nonzero value
// to a nonzero value of the same sign).  The rounded quotient underflows to 0
// for a positive r below 2^-1075 and would take the r <= 0 branch, or
// overflows to +-inf.  Ties go to the lower branch, as in psi_branch.  r (the
// rounded quotient) serves van Leer's smooth derivative only.
double dpsi_exact(int lim, double dU, double du, double r) {
  const double q = std::fabs(du);
  const double p = std::signbit(du) ? -dU : dU;
  if (lim == L_UPWIND || lim == L_CENTRAL || p <= 0.0) return 0.0;
  switch (lim) {
    case L_MINMOD: return (p - q <= 0.0) ? 1.0 : 0.0;                 // r <= 1
    case L_VANLEER: return std::isinf(r) ? 0.0 : 2.0 / ((1.0 + r) * (1.0 + r));
    case L_SUPERBEE:
      if (std::fma(2.0, p, -q) <= 0.0) return 2.0;                    // r <= 1/2
      if (p - q <= 0.0) return 0.0;                                   // r <= 1
      if (std::fma(-2.0, q, p) <= 0.0) return 1.0;                    // r <= 2
      return 0.0;
    case L_SMART:
      if (std::fma(5.0, p, -q) <= 0.0) return 2.0;                    // r <= 1/5
      if (std::fma(-5.0, q, p) <= 0.0) return 0.75;                   // r <= 5
      return 0.0;
  }
  return std::nan("");
}

// ------------------------------------------------------------ one face
struct FaceEval {
  int s;            // +1 / -1
  int32_t C, D, U;  // centred, downwind, upstream cell (U = -1 if not unique)
  double du, dU;    // Delta_u theta, Delta_U theta
  double r;         // gradient ratio (NaN when du == 0)
  double thf;       // limited face value
  double psi, dpsi; // limiter value and branch derivative (when du != 0)
};

// The upwind side: eq. (sign) with Table 1's x > 0 ? +1 : -1.
inline int face_sign(double u) { return (u > 0.0) ? 1 : -1; }

FaceEval eval_face(const OMesh &m, int lim, const double *th, const double *u, int64_t f) {
  FaceEval e;
  e.s = face_sign(u[f]);
  const int32_t a = m.c0[f], b = m.c1[f];
  e.C = (e.s > 0) ? a : b;
  e.D = (e.s > 0) ? b : a;
  // eq. (Delta_face): difference across f taken along the flow.
  e.du = th[e.D] - th[e.C];
  // eq. (Delta_Upwind), sign-corrected: other faces of C projected on n_f.
  double acc = 0.0;
  int32_t U = -1;
  int n_nonzero = 0;
  for (int64_t q = m.cf_ptr[e.C]; q < m.cf_ptr[e.C + 1]; ++q) {
    const int64_t j = m.cf_idx[q];
    if (j == f) continue;
    const double w = m.nx[f] * m.nx[j] + m.ny[f] * m.ny[j] + m.nz[f] * m.nz[j];
    acc = acc + dist_term(m, w * (th[m.c1[j]] - th[m.c0[j]]), j);
    if (w != 0.0) {
      ++n_nonzero;
      U = (m.c0[j] == e.C) ? m.c1[j] : m.c0[j];
    }
  }
  e.U = (n_nonzero == 1) ? U : -1;
  acc = dist_face(m, acc, f);
  e.dU = (e.s > 0) ? acc : -acc;
  // eq. (rf) and eq. (FL-UP); a zero denominator keeps the upwind value.
  // Psi there is 0 (the upwind side of the kink at d_u = 0), except for the
  // central reconstruction, whose Psi = 1 does not depend on r: its face
  // value theta_C + d_u / 2 is linear through d_u = 0 (eq. FL-CD with F = 0),
  // and the tangent-linear model takes that slope.
  if (e.du == 0.0) {
    e.r = std::nan("");
    e.psi = (lim == L_CENTRAL) ? 1.0 : 0.0;
    e.dpsi = 0.0;
    e.thf = th[e.C];
  } else {
    e.r = e.dU / e.du;
    e.psi = psi_closed(lim, e.r);
    e.dpsi = dpsi_exact(lim, e.dU, e.du, e.r);
    e.thf = th[e.C] + 0.5 * e.psi * e.du;
  }
  return e;
}

// R(theta): Algorithm 4's dt-free increment, M U(u_f) theta_f.
void rhs(const OMesh &m, int lim, const double *th, const double *u, double *R,
         double *phi_scratch) {
  const int64_t F = m.F, C = m.C;
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < F; ++f) {
    FaceEval e = eval_face(m, lim, th, u, f);
    phi_scratch[f] = u[f] * m.area[f] * e.thf;
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < C; ++c) {
    double acc = 0.0;
    for (int64_t q = m.cf_ptr[c]; q < m.cf_ptr[c + 1]; ++q) {
      const int64_t f = m.cf_idx[q];
      const double sigma = (m.c0[f] == c) ? 1.0 : -1.0;
      // a face whose two cells coincide contributes +phi - phi = 0
      if (m.c0[f] == m.c1[f]) continue;
      acc = acc + sigma * phi_scratch[f];
    }
    R[c] = -acc / m.vol[c];
  }
}

// Coefficient of d(d_u) in the tangent-linear face value, (Psi - Psi' r)/2.
// On a branch where Psi is constant (Psi' = 0) theta_f = theta_C + Psi d_u/2
// is linear in d_u with slope Psi/2 for every r, r = +-inf included (a
// subnormal d_u beside a normal d_U overflows r): the product Psi' r is zero
// there, not 0 * inf.
inline double tlm_alpha(const FaceEval &e) {
  const double pr = (e.dpsi != 0.0) ? e.dpsi * e.r : 0.0;
  return 0.5 * (e.psi - pr);
}

// Tangent-linear of theta_f: returns d theta_f for input perturbation dth.
double face_tlm(const OMesh &m, const FaceEval &e, const double *dth, int64_t f) {
  const double ddu = dth[e.D] - dth[e.C];
  double acc = 0.0;
  for (int64_t q = m.cf_ptr[e.C]; q < m.cf_ptr[e.C + 1]; ++q) {
    const int64_t j = m.cf_idx[q];
    if (j == f) continue;
    const double w = m.nx[f] * m.nx[j] + m.ny[f] * m.ny[j] + m.nz[f] * m.nz[j];
    acc = acc + dist_term(m, w * (dth[m.c1[j]] - dth[m.c0[j]]), j);
  }
  acc = dist_face(m, acc, f);
  const double ddU = (e.s > 0) ? acc : -acc;
  if (e.du == 0.0) return dth[e.C] + 0.5 * e.psi * ddu;
  // theta_f = theta_C + Psi(r) du / 2, r = dU / du
  //   d theta_f = d theta_C + (Psi - Psi' r)/2 d du + Psi'/2 d dU
  const double alpha = tlm_alpha(e);
  const double beta = 0.5 * e.dpsi;
  return dth[e.C] + alpha * ddu + beta * ddU;
}

void rhs_tlm(const OMesh &m, int lim, const double *th, const double *dth, const double *u,
             double *dR, double *scratch) {
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < m.F; ++f) {
    FaceEval e = eval_face(m, lim, th, u, f);
    scratch[f] = u[f] * m.area[f] * face_tlm(m, e, dth, f);
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < m.C; ++c) {
    double acc = 0.0;
    for (int64_t q = m.cf_ptr[c]; q < m.cf_ptr[c + 1]; ++q) {
      const int64_t f = m.cf_idx[q];
      if (m.c0[f] == m.c1[f]) continue;
      const double sigma = (m.c0[f] == c) ? 1.0 : -1.0;
      acc = acc + sigma * scratch[f];
    }
    dR[c] = -acc / m.vol[c];
  }
}

// Transpose of d R / d theta applied to mu (sequential scatter, face order).
void rhs_adjoint(const OMesh &m, int lim, const double *th, const double *u, const double *mu,
                 double *out) {
  for (int64_t c = 0; c < m.C; ++c) out[c] = 0.0;
  for (int64_t f = 0; f < m.F; ++f) {
    if (m.c0[f] == m.c1[f]) continue;
    FaceEval e = eval_face(m, lim, th, u, f);
    // R_c0 gets -phi/V_c0, R_c1 gets +phi/V_c1
    const double g = u[f] * m.area[f] * (mu[m.c1[f]] / m.vol[m.c1[f]] - mu[m.c0[f]] / m.vol[m.c0[f]]);
    if (e.du == 0.0) {
      out[e.C] += g * (1.0 - 0.5 * e.psi);
      out[e.D] += g * (0.5 * e.psi);
      continue;
    }
    const double alpha = tlm_alpha(e);
    const double beta = 0.5 * e.dpsi;
    out[e.C] += g * (1.0 - alpha);
    out[e.D] += g * alpha;
    const double gb = (e.s > 0) ? g * beta : -(g * beta);
    for (int64_t q = m.cf_ptr[e.C]; q < m.cf_ptr[e.C + 1]; ++q) {
      const int64_t j = m.cf_idx[q];
      if (j == f) continue;
      const double w = m.nx[f] * m.nx[j] + m.ny[f] * m.ny[j] + m.nz[f] * m.nz[j];
      if (w == 0.0) continue;
      // d(d_U)/d(theta) of the weighted sum: w d_f / d_j per term
      const double wj = dist_face(m, dist_term(m, w, j), f);
      out[m.c1[j]] += gb * wj;
      out[m.c0[j]] -= gb * wj;
    }
  }
}

// SSP-RK3 stage coefficients: y = a * theta^n + b * (x + dt R(x)).
const double RK3_A[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK3_B[3] = {1.0, 0.25, 2.0 / 3.0};

void stage(const OMesh &m, int lim, int rk, int st, double dt, const double *thn, const double *x,
           const double *u, double *y, double *R, double *scratch) {
  rhs(m, lim, x, u, R, scratch);
  if (rk == 1) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m.C; ++c) y[c] = x[c] + dt * R[c];
  } else if (st == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m.C; ++c) y[c] = thn[c] + dt * R[c];
  } else {
    const double a = RK3_A[st], b = RK3_B[st];
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m.C; ++c) y[c] = a * thn[c] + b * (x[c] + dt * R[c]);
  }
}

thread_local char g_err[256] = "";
void set_err(const char *msg) { std::strncpy(g_err, msg, sizeof(g_err) - 1); }

}  // namespace

extern "C" {

const char *orc_last_error(void) { return g_err; }

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// Builds the oracle's own face/cell tables.  Returns NULL on invalid input.
void *orc_mesh_new(int64_t C, int64_t F, const int32_t *face_cells, const double *normals,
                   const double *areas, const double *volumes) {
  if (C < 0 || F < 0) { set_err("negative size"); return nullptr; }
  OMesh *m = new OMesh();
  m->C = C;
  m->F = F;
  m->c0.resize(F); m->c1.resize(F);
  m->nx.resize(F); m->ny.resize(F); m->nz.resize(F);
  m->area.assign(areas, areas + F);
  m->vol.assign(volumes, volumes + C);
  std::vector<int64_t> deg(C + 1, 0);
  for (int64_t f = 0; f < F; ++f) {
    const int32_t a = face_cells[2 * f], b = face_cells[2 * f + 1];
    if (a < 0 || b < 0 || a >= C || b >= C) { set_err("face cell out of range"); delete m; return nullptr; }
    m->c0[f] = a; m->c1[f] = b;
    m->nx[f] = normals[3 * f]; m->ny[f] = normals[3 * f + 1]; m->nz[f] = normals[3 * f + 2];
    deg[a]++;
    if (b != a) deg[b]++;
  }
  m->cf_ptr.assign(C + 1, 0);
  for (int64_t c = 0; c < C; ++c) m->cf_ptr[c + 1] = m->cf_ptr[c] + deg[c];
  m->cf_idx.assign(m->cf_ptr[C], 0);
  std::vector<int64_t> fill(m->cf_ptr.begin(), m->cf_ptr.end() - 1);
  for (int64_t f = 0; f < F; ++f) {  // ascending f => each list is sorted
    m->cf_idx[fill[m->c0[f]]++] = f;
    if (m->c1[f] != m->c0[f]) m->cf_idx[fill[m->c1[f]]++] = f;
  }
  return m;
}

// Face distances d_f (distance between the centres of c0 and c1, > 0) of a
// non-uniform mesh; NULL removes them (uniform spacing, no weights).
int orc_mesh_set_distances(void *h, const double *d) {
  OMesh &m = *static_cast<OMesh *>(h);
  if (d == nullptr) {
    m.dist.clear();
    return 0;
  }
  for (int64_t f = 0; f < m.F; ++f)
    if (!(d[f] > 0.0) || !std::isfinite(d[f])) { set_err("face distances must be > 0"); return 1; }
  m.dist.assign(d, d + m.F);
  return 0;
}

void orc_mesh_free(void *h) { delete static_cast<OMesh *>(h); }

int orc_psi(int lim, const double *r, double *psi, int64_t n) {
  for (int64_t i = 0; i < n; ++i) psi[i] = psi_closed(lim, r[i]);
  return 0;
}

int orc_psi_branch(int lim, const double *r, double *psi, double *dpsi, int64_t n) {
  for (int64_t i = 0; i < n; ++i) psi[i] = psi_branch(lim, r[i], &dpsi[i]);
  return 0;
}

// Algorithm 1's output theta_f plus the per-face selection (s, C, D, U) and
// the two differences.  Any output pointer may be NULL.
int orc_face_values(const void *h, int lim, const double *th, const double *u, double *thf,
                    int32_t *sel /*[F][4] s,C,D,U*/, double *du, double *dU) {
  const OMesh &m = *static_cast<const OMesh *>(h);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < m.F; ++f) {
    FaceEval e = eval_face(m, lim, th, u, f);
    if (thf) thf[f] = e.thf;
    if (sel) { sel[4 * f] = e.s; sel[4 * f + 1] = e.C; sel[4 * f + 2] = e.D; sel[4 * f + 3] = e.U; }
    if (du) du[f] = e.du;
    if (dU) dU[f] = e.dU;
  }
  return 0;
}

int orc_rhs(const void *h, int lim, const double *th, const double *u, double *R) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  std::vector<double> scratch(m.F);
  rhs(m, lim, th, u, R, scratch.data());
  return 0;
}

// nsteps explicit steps, in place.  rk = 1 (forward Euler, Algorithm 4) or 3.
int orc_step(const void *h, int lim, int rk, double dt, int64_t nsteps, const double *u,
             double *th) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  if (rk != 1 && rk != 3) { set_err("rk must be 1 or 3"); return 1; }
  std::vector<double> thn(m.C), a(m.C), b(m.C), R(m.C), scratch(m.F);
  for (int64_t n = 0; n < nsteps; ++n) {
    std::memcpy(thn.data(), th, sizeof(double) * m.C);
    if (rk == 1) {
      stage(m, lim, 1, 0, dt, thn.data(), thn.data(), u, th, R.data(), scratch.data());
    } else {
      stage(m, lim, 3, 0, dt, thn.data(), thn.data(), u, a.data(), R.data(), scratch.data());
      stage(m, lim, 3, 1, dt, thn.data(), a.data(), u, b.data(), R.data(), scratch.data());
      stage(m, lim, 3, 2, dt, thn.data(), b.data(), u, th, R.data(), scratch.data());
    }
  }
  return 0;
}

// nsteps steps with a time-modulated velocity: stage s of step n uses the
// face velocity g[n * S + s] * u_f (S = 1 for Euler, 3 for SSP-RK3), the form
// of the reversing deformation flow of Section 4.1 (eq. rhodonea), whose
// velocity is a fixed field times cos(pi t / T).  Everything else is orc_step.
int orc_step_modulated(const void *h, int lim, int rk, double dt, int64_t nsteps, const double *u,
                       const double *g, double *th) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  if (rk != 1 && rk != 3) { set_err("rk must be 1 or 3"); return 1; }
  const int S = (rk == 1) ? 1 : 3;
  std::vector<double> thn(m.C), a(m.C), b(m.C), R(m.C), scratch(m.F), us(m.F);
  auto scaled = [&](int64_t n, int st) {
    const double gs = g[n * S + st];
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < m.F; ++f) us[f] = gs * u[f];
    return us.data();
  };
  for (int64_t n = 0; n < nsteps; ++n) {
    std::memcpy(thn.data(), th, sizeof(double) * m.C);
    if (rk == 1) {
      stage(m, lim, 1, 0, dt, thn.data(), thn.data(), scaled(n, 0), th, R.data(), scratch.data());
    } else {
      stage(m, lim, 3, 0, dt, thn.data(), thn.data(), scaled(n, 0), a.data(), R.data(), scratch.data());
      stage(m, lim, 3, 1, dt, thn.data(), a.data(), scaled(n, 1), b.data(), R.data(), scratch.data());
      stage(m, lim, 3, 2, dt, thn.data(), b.data(), scaled(n, 2), th, R.data(), scratch.data());
    }
  }
  return 0;
}

// One RK stage: y = a*thn + b*(x + dt R(x)) with (a, b) of stage st.
int orc_stage(const void *h, int lim, int rk, int st, double dt, const double *thn, const double *x,
              const double *u, double *y) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  std::vector<double> R(m.C), scratch(m.F);
  stage(m, lim, rk, st, dt, thn, x, u, y, R.data(), scratch.data());
  return 0;
}

// Tangent-linear rollout: advances (theta, dtheta) together for nsteps.
int orc_step_tlm(const void *h, int lim, int rk, double dt, int64_t nsteps, const double *u,
                 double *th, double *dth) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  if (rk != 1 && rk != 3) { set_err("rk must be 1 or 3"); return 1; }
  const int ns = (rk == 1) ? 1 : 3;
  std::vector<double> thn(m.C), dthn(m.C), x(m.C), dx(m.C), y(m.C), dy(m.C), R(m.C), dR(m.C),
      scratch(m.F);
  for (int64_t n = 0; n < nsteps; ++n) {
    std::memcpy(thn.data(), th, sizeof(double) * m.C);
    std::memcpy(dthn.data(), dth, sizeof(double) * m.C);
    x = thn;
    dx = dthn;
    for (int st = 0; st < ns; ++st) {
      rhs(m, lim, x.data(), u, R.data(), scratch.data());
      rhs_tlm(m, lim, x.data(), dx.data(), u, dR.data(), scratch.data());
      const double a = (rk == 1) ? 0.0 : RK3_A[st], b = (rk == 1) ? 1.0 : RK3_B[st];
      for (int64_t c = 0; c < m.C; ++c) {
        if (st == 0) {
          y[c] = thn[c] + dt * R[c];
          dy[c] = dthn[c] + dt * dR[c];
        } else {
          y[c] = a * thn[c] + b * (x[c] + dt * R[c]);
          dy[c] = a * dthn[c] + b * (dx[c] + dt * dR[c]);
        }
      }
      x.swap(y);
      dx.swap(dy);
    }
    std::memcpy(th, x.data(), sizeof(double) * m.C);
    std::memcpy(dth, dx.data(), sizeof(double) * m.C);
  }
  return 0;
}

// Transpose of d(R)/d(theta) at theta applied to mu (one operator).
int orc_rhs_adjoint(const void *h, int lim, const double *th, const double *u, const double *mu,
                    double *out) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  rhs_adjoint(m, lim, th, u, mu, out);
  return 0;
}

// Gradient of J = 0.5 ||theta_T - target||^2 with respect to theta_0, by
// storing every stage input of the rollout and sweeping the stages backwards.
// Also returns J.  Memory: nsteps * stages * C doubles.
int orc_gradient(const void *h, int lim, int rk, double dt, int64_t nsteps, const double *u,
                 const double *th0, const double *target, double *grad, double *J) {
  const OMesh &m = *static_cast<const OMesh *>(h);
  if (rk != 1 && rk != 3) { set_err("rk must be 1 or 3"); return 1; }
  const int ns = (rk == 1) ? 1 : 3;
  const int64_t C = m.C;
  std::vector<double> store((size_t)(nsteps * ns) * C);  // stage inputs x
  std::vector<double> thn(th0, th0 + C), y(C), R(C), scratch(m.F), x(C);
  std::vector<double> hist_n((size_t)nsteps * C);         // theta^n of each step
  for (int64_t n = 0; n < nsteps; ++n) {
    std::memcpy(&hist_n[(size_t)n * C], thn.data(), sizeof(double) * C);
    x = thn;
    for (int st = 0; st < ns; ++st) {
      std::memcpy(&store[((size_t)n * ns + st) * C], x.data(), sizeof(double) * C);
      stage(m, lim, rk, st, dt, thn.data(), x.data(), u, y.data(), R.data(), scratch.data());
      x.swap(y);
    }
    thn = x;
  }
  double j = 0.0;
  std::vector<double> lam(C);  // adjoint of theta_T
  for (int64_t c = 0; c < C; ++c) {
    const double d = thn[c] - target[c];
    j += 0.5 * d * d;
    lam[c] = d;
  }
  if (J) *J = j;
  std::vector<double> lam_n(C), lam_x(C), tmp(C);
  for (int64_t n = nsteps - 1; n >= 0; --n) {
    // lam is the adjoint of the last stage output; theta^n enters every stage
    std::fill(lam_n.begin(), lam_n.end(), 0.0);
    for (int st = ns - 1; st >= 0; --st) {
      const double *xs = &store[((size_t)n * ns + st) * C];
      const double a = (rk == 1 || st == 0) ? 0.0 : RK3_A[st];
      const double b = (rk == 1 || st == 0) ? 1.0 : RK3_B[st];
      rhs_adjoint(m, lim, xs, u, lam.data(), tmp.data());
      for (int64_t c = 0; c < C; ++c) {
        // y = a thn + b (x + dt R(x))  (stage 0 of RK3: y = thn + dt R(thn), x == thn)
        lam_n[c] += a * lam[c];
        lam_x[c] = b * lam[c] + b * dt * tmp[c];
      }
      lam.swap(lam_x);
    }
    // stage 0's input is theta^n itself
    for (int64_t c = 0; c < C; ++c) lam[c] += lam_n[c];
  }
  std::memcpy(grad, lam.data(), sizeof(double) * C);
  return 0;
}

}  // extern "C"
