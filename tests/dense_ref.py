"""Brute-force dense reference for the oracle pins (tests only).

Everything here is built from the polynomial definitions with numpy, with no
code shared with the oracle's tensor loops: the Lagrange basis of the GLL
nodes as numpy polynomials, D from differentiating them, quadrature weights
from integrating them exactly, element operators as explicit Kronecker
products, Jacobians by numpy determinant/inverse, and assembly with an explicit
scatter matrix Q (Sec. II-A: u_L = Q u, A = QQ^T A_L).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import Polynomial

import workloads as W


def lagrange_basis(xi: np.ndarray):
    """Lagrange polynomials l_j with l_j(xi_m) = delta_jm."""
    out = []
    for j in range(len(xi)):
        p = Polynomial([1.0])
        for m in range(len(xi)):
            if m != j:
                p = p * Polynomial([-xi[m], 1.0]) / (xi[j] - xi[m])
        out.append(p)
    return out


def basis_data(N: int):
    """(xi, rho, D) of order N: nodes from numpy's Legendre roots, weights as
    exact integrals of the Lagrange basis, D[i, j] = l_j'(xi_i)."""
    xi = W.gll_positions(N)
    ls = lagrange_basis(xi)
    rho = np.array([l.integ()(1.0) - l.integ()(-1.0) for l in ls])
    D = np.array([[ls[j].deriv()(xi[i]) for j in range(N + 1)] for i in range(N + 1)])
    return xi, rho, D


def stiffness_1d_exact(N: int) -> np.ndarray:
    """K_ij = int_{-1}^{1} l_i' l_j' dx by exact polynomial integration."""
    xi = W.gll_positions(N)
    ls = [l.deriv() for l in lagrange_basis(xi)]
    K = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            q = (ls[i] * ls[j]).integ()
            K[i, j] = q(1.0) - q(-1.0)
    return K


def derivative_matrices(D: np.ndarray):
    """Dense (lx^3 x lx^3) derivative operators along r (i), s (j), t (k) for
    vectors with i fastest."""
    lx = D.shape[0]
    I = np.eye(lx)
    Dr = np.kron(I, np.kron(I, D))
    Ds = np.kron(I, np.kron(D, I))
    Dt = np.kron(D, np.kron(I, I))
    return Dr, Ds, Dt


def element_matrices(mesh, h1=None):
    """Dense A^e = sum_st D_s^T diag(h1 G_st) D_t for every element, with G from
    numpy Jacobians.  Returns (A_e [E, n3, n3], B [E, n3])."""
    N = mesh.N
    lx = mesh.lx
    n3 = lx ** 3
    _, rho, D = basis_data(N)
    Dr, Ds, Dt = derivative_matrices(D)
    w3 = np.kron(rho, np.kron(rho, rho))
    Ds_ = [Dr, Ds, Dt]
    out = np.zeros((mesh.E, n3, n3))
    Bm = np.zeros((mesh.E, n3))
    hh = np.ones(mesh.n_local) if h1 is None else np.asarray(h1)
    for e in range(mesh.E):
        X = mesh.coords[:, e, :]  # [3, n3]
        Jm = np.zeros((n3, 3, 3))
        for m in range(3):
            for s in range(3):
                Jm[:, m, s] = Ds_[s] @ X[m]
        J = np.linalg.det(Jm)
        inv = np.linalg.inv(Jm)  # inv[q, s, l] = dr_s/dx_l
        he = hh[e * n3:(e + 1) * n3]
        A = np.zeros((n3, n3))
        for s in range(3):
            for t in range(3):
                g = w3 * J * np.einsum("ql,ql->q", inv[:, s, :], inv[:, t, :]) * he
                A += Ds_[s].T @ (g[:, None] * Ds_[t])
        out[e] = A
        Bm[e] = w3 * J
    return out, Bm


def element_magnitude_matrices(mesh, h1=None):
    """Dense sum_st |D_s|^T diag(|h1 G_st|) |D_t| per element: the magnitudes
    of the terms of A^e u act on |u| through this nonnegative matrix."""
    N = mesh.N
    lx = mesh.lx
    n3 = lx ** 3
    _, rho, D = basis_data(N)
    Ds_ = [np.abs(M) for M in derivative_matrices(D)]
    Dsigned = derivative_matrices(D)
    w3 = np.kron(rho, np.kron(rho, rho))
    hh = np.ones(mesh.n_local) if h1 is None else np.asarray(h1)
    out = np.zeros((mesh.E, n3, n3))
    for e in range(mesh.E):
        X = mesh.coords[:, e, :]
        Jm = np.zeros((n3, 3, 3))
        for m in range(3):
            for s in range(3):
                Jm[:, m, s] = Dsigned[s] @ X[m]
        J = np.linalg.det(Jm)
        inv = np.linalg.inv(Jm)
        he = hh[e * n3:(e + 1) * n3]
        A = np.zeros((n3, n3))
        for s in range(3):
            for t in range(3):
                g = np.abs(w3 * J * np.einsum("ql,ql->q", inv[:, s, :], inv[:, t, :]) * he)
                A += Ds_[s].T @ (g[:, None] * Ds_[t])
        out[e] = A
    return out


def scatter_matrix(mesh):
    """Q (n_L x n_U) with Q[L, g] = 1 when local node L is a copy of global node g
    (global nodes numbered by ascending id).  Also returns the mask per global node."""
    ug, inv = np.unique(mesh.gid, return_inverse=True)
    Q = np.zeros((mesh.n_local, ug.shape[0]))
    Q[np.arange(mesh.n_local), inv] = 1.0
    mask_g = np.zeros(ug.shape[0])
    mask_g[inv] = mesh.mask
    return Q, mask_g, inv


def assembled(mesh, h1=None):
    """Dense assembled stiffness K = Q^T A_L Q and mass b = Q^T B (n_U)."""
    Ae, Bm = element_matrices(mesh, h1)
    n3 = mesh.lx ** 3
    Q, mask_g, inv = scatter_matrix(mesh)
    K = np.zeros((Q.shape[1], Q.shape[1]))
    for e in range(mesh.E):
        Qe = Q[e * n3:(e + 1) * n3]
        K += Qe.T @ Ae[e] @ Qe
    return K, Q, mask_g, Ae, Bm
