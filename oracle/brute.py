"""Dense-matrix brute force of the paper's algebraic formulation (TEST
INFRASTRUCTURE ONLY; tiny meshes).

Every operator is assembled as a dense NumPy matrix straight from its
definition, then Algorithm 1 / Algorithm 4 are evaluated as matrix-vector
products.  This is independent of the stencil oracle in ``fl_oracle.cpp``:
it never looks up an upstream cell, it only multiplies matrices.

Definitions (Valle et al., Sections 2-3):

* E = T_{C->F}, |F| x |C| directed incidence: E[f, c0] = -1, E[f, c1] = +1
  (eq. Tfc; the normal of f points from c0 to c1).
* B = |E| (eq. UnOrInMatrix), W_FF = diag(B 1) (eq. DegMatrix),
  Pi_{C->F} = W^-1 B (eq. sCF).
* A_FF = B B^T - W (eq. AdjacencyFaces; printed as W - B B^T, read with the
  sign that makes the entries non-negative and reproduces the printed
  example matrix ADJM).
* D^A_FF = offdiag(E B^T) (eq. DirectedAdjacencyFaces).
* N = (N_1 | ... | N_d), N_a = diag(n_a) (eq. normal).
* Q = diag(u > 0 ? +1 : -1) (eq. sign; Table 1 signxty).
* S = 1/2 N (I_d (x) D^A) N^T E,  T = 1/2 N (I_d (x) A) N^T E (the two
  precomputed matrices after eq. SimplifiedDeltaUpstream).
* d_u = Q E theta (eq. Delta_face).
* d_U = Q N (I_d (x) A^U) N^T E theta with A^U = 1/2 (A - Q D^A)
  (eq. Delta_Upwind, eq. UpstreamAdjacency), which expands to
  d_U = (Q T - S) theta.  The extra left factor Q is the sign correction
  (without it the upstream difference has the wrong sign whenever the flow
  runs against the face normal).
* theta_f = (Pi + F(r) Q E) theta = Pi theta + F(r) d_u, F = (Psi - 1)/2
  (eq. FL-operator), r = d_U / d_u (eq. rf).
* M = V^-1 E^T diag(A_f): theta^{n+1} = theta^n + dt M U(u_f) theta_f
  (Algorithm 4, with M read as minus the divergence).
"""
from __future__ import annotations

import numpy as np


def psi_np(lim: str, r):
    """Limiter closed forms, evaluated independently of the C++ oracle."""
    r = np.asarray(r, dtype=np.float64)
    if lim == "upwind":
        return np.zeros_like(r)
    if lim == "central":
        return np.ones_like(r)
    if lim == "minmod":
        return np.maximum(0.0, np.minimum(1.0, r))
    if lim == "superbee":
        return np.maximum(0.0, np.maximum(np.minimum(1.0, 2.0 * r), np.minimum(r, 2.0)))
    if lim == "smart":
        return np.maximum(0.0, np.minimum(np.minimum(2.0 * r, 0.25 + 0.75 * r), 4.0))
    if lim == "vanleer":
        out = np.zeros_like(r)
        pos = r > 0
        rp = r[pos]
        out[pos] = np.where(np.isinf(rp), 2.0, (rp + np.abs(rp)) / (1.0 + np.abs(rp)))
        return out
    raise ValueError(lim)


def incidence(face_cells, n_cells):
    F = face_cells.shape[0]
    E = np.zeros((F, n_cells))
    for f, (a, b) in enumerate(face_cells):
        E[f, a] += -1.0
        E[f, b] += 1.0
    return E


def topology(E):
    """B, W_FF, Pi, A_FF, D^A_FF from a directed incidence matrix."""
    B = np.abs(E)
    W = np.diag(B @ np.ones(B.shape[1]))
    Pi = np.linalg.inv(W) @ B
    A = B @ B.T - W
    DA = E @ B.T
    DA = DA - np.diag(np.diag(DA))
    return B, W, Pi, A, DA


def normal_matrix(normals):
    F = normals.shape[0]
    d = normals.shape[1]
    return np.hstack([np.diag(normals[:, a]) for a in range(d)]), d


def operators(mesh):
    E = incidence(np.asarray(mesh.face_cells), mesh.n_cells)
    B, W, Pi, A, DA = topology(E)
    N, d = normal_matrix(np.asarray(mesh.normals))
    I = np.eye(d)
    S = 0.5 * N @ np.kron(I, DA) @ N.T @ E
    T = 0.5 * N @ np.kron(I, A) @ N.T @ E
    M = np.diag(1.0 / np.asarray(mesh.volumes)) @ E.T @ np.diag(np.asarray(mesh.areas))
    return {"E": E, "B": B, "W": W, "Pi": Pi, "A": A, "DA": DA, "N": N, "S": S, "T": T, "M": M,
            "d": d}


def sign_matrix(u):
    return np.diag(np.where(np.asarray(u) > 0, 1.0, -1.0))


def face_values(ops, lim, theta, u):
    """Algorithm 1 with the corrected upstream difference.  Returns theta_f,
    d_u, d_U.  A zero denominator keeps the centred (upwind) value, i.e.
    theta_f = Pi theta - d_u / 2 there (F = -1/2, Psi = 0)."""
    Q = sign_matrix(u)
    E, S, T, Pi = ops["E"], ops["S"], ops["T"], ops["Pi"]
    du = Q @ E @ theta
    dU = (Q @ T - S) @ theta
    with np.errstate(divide="ignore", invalid="ignore"):
        r = dU / du
    psi = np.where(du == 0, 0.0, psi_np(lim, np.where(du == 0, 0.0, r)))
    Fdiag = (psi - 1.0) / 2.0
    thf = Pi @ theta + Fdiag * du
    return thf, du, dU


def selection(ops, u):
    """Upwind (C), downwind (D) and upstream (U) cells read off the matrices:
    C/D from the rows of Q E, U from the rows of Q N (I (x) A^U) N^T E, whose
    only nonzero entries on a hexahedral mesh are +1 at C and -1 at U."""
    Q = sign_matrix(u)
    E = ops["E"]
    QE = Q @ E
    C = np.argmin(QE, axis=1)
    D = np.argmax(QE, axis=1)
    AU = 0.5 * (ops["A"] - Q @ ops["DA"])
    G = Q @ ops["N"] @ np.kron(np.eye(ops["d"]), AU) @ ops["N"].T @ E
    U = np.full(E.shape[0], -1)
    for f in range(E.shape[0]):
        neg = np.nonzero(G[f] < -0.5)[0]
        if len(neg) == 1:
            U[f] = neg[0]
    return C, D, U


def rhs(ops, lim, theta, u):
    thf, _, _ = face_values(ops, lim, theta, u)
    return ops["M"] @ (np.asarray(u) * thf)


def step(ops, lim, rk, dt, nsteps, u, theta):
    th = np.array(theta, dtype=np.float64)
    for _ in range(nsteps):
        if rk == 1:
            th = th + dt * rhs(ops, lim, th, u)
        else:
            a = th + dt * rhs(ops, lim, th, u)
            b = 0.75 * th + 0.25 * (a + dt * rhs(ops, lim, a, u))
            th = th / 3.0 + (2.0 / 3.0) * (b + dt * rhs(ops, lim, b, u))
    return th
