"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake (a transposed operand, a dropped term, a wrong
sign or index, a wrong weight) into a COPY of the oracle's C source, builds it
on the CPU, and checks that the pin battery below fails for it while passing
for the unmodified oracle."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W
import dense_ref

SRC = os.path.join(os.path.dirname(oracle.__file__), "sem_oracle.c")

MUTANTS = {
    "transposed_D_in_backward_contraction": (
        "acc += p->D[l * lx + i] * ur[", "acc += p->D[i * lx + l] * ur["),
    "dropped_G12_term": (
        "ur[q] = h * (g11 * a + g12 * b + g13 * c);", "ur[q] = h * (g11 * a + g13 * c);"),
    "wrong_sign_inverse_jacobian": (
        "inv[0][1] = (cc * h - b * kk) / J;", "inv[0][1] = (b * kk - cc * h) / J;"),
    "gll_weight_missing_square": (
        "rho[i] = (double)(2.0L / ((long double)N * (N + 1) * pN * pN));",
        "rho[i] = (double)(2.0L / ((long double)N * (N + 1) * pN));"),
    "gs_skips_last_copy": (
        "for (int64_t c = p->grp[g]; c < p->grp[g + 1]; c++) s += u[p->order[c]];",
        "for (int64_t c = p->grp[g]; c < p->grp[g + 1] - 1; c++) s += u[p->order[c]];"),
    "jacobi_cross_term_factor": ("s += 2.0 * p->h1[L] *", "s += p->h1[L] *"),
    "cg_beta_inverted": (
        "const double beta = (it == 0) ? 0.0 : rho / rho_old;",
        "const double beta = (it == 0) ? 0.0 : rho_old / rho;"),
    "dot_without_multiplicity": (
        "for (int64_t L = 0; L < p->n; L++) s += a[L] * b[L] / p->mult[L];",
        "for (int64_t L = 0; L < p->n; L++) s += a[L] * b[L];"),
    "dmat_corner_sign": (
        "else if (i == 0) v = -(long double)N * (N + 1) / 4.0L;",
        "else if (i == 0) v = (long double)N * (N + 1) / 4.0L;"),
    "jacobian_index_s_uses_k": (
        "d[m][1] += p->D[j * lx + l] * c[m][k * lx * lx + l * lx + i];",
        "d[m][1] += p->D[k * lx + l] * c[m][k * lx * lx + l * lx + i];"),
    "h1_at_wrong_point_in_jacobi": (
        "s += D[l * lx + i] * D[l * lx + i] * p->h1[La] * p->G[0 * n + La];",
        "s += D[l * lx + i] * D[l * lx + i] * p->h1[L0] * p->G[0 * n + La];"),
    "ir_kept_direction_rescaled_by_c_squared": (
        "rho_carry * (rn_prev / rn) : 0.0;", "rho_carry * (rn_prev / rn) * (rn_prev / rn) : 0.0;"),
    "helmholtz_mass_without_jacobian_weights": (
        "if (p->h2) acc += p->h2[L] * p->B[L] * ue[k * lx * lx + j * lx + i];",
        "if (p->h2) acc += p->h2[L] * ue[k * lx * lx + j * lx + i];"),
    "helmholtz_jacobi_without_mass_term": (
        "if (p->h2) s += p->h2[L] * p->B[L];", ""),
    "ir_kept_direction_rescaled_by_inverse": (
        "rho_carry * (rn_prev / rn) : 0.0;", "rho_carry * (rn / rn_prev) : 0.0;"),
}


def _battery() -> list[str]:
    """Run a compact set of the oracle pins; return the names of failed pins."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    for N in (2, 4):
        xi, rho = oracle.gll(N)
        check("gll_sum", abs(rho.sum() - 2) < 1e-14)
        D = oracle.dmat(N)
        check("dmat_poly", all(np.max(np.abs(D @ xi ** m - m * xi ** max(m - 1, 0))) < 1e-12
                               for m in range(1, N + 1)))
        xr, rr, Dr = dense_ref.basis_data(N)
        check("gll_vs_lagrange", np.allclose(rho, rr, rtol=1e-12) and np.allclose(D, Dr, atol=1e-11))
    # dense brute force on a deformed mesh with h1
    # jittered nodes: the geometric factors differ between the copies of a node, so
    # the cross terms of the Jacobi diagonal do not cancel in the assembly
    m = W.box_mesh(3, 2, 2, 2, amp=0.1, jitter=0.03, seed=5)
    h1 = W.h1_wavy(m)
    try:
        P = oracle.Problem(m, h1)
    except ValueError:
        return ["setup_rejected"]
    K, Q, mask_g, Ae, Bm = dense_ref.assembled(m, h1)
    rng = np.random.default_rng(0)
    ug = rng.standard_normal(Q.shape[1])
    ref = Q @ (mask_g * (K @ ug))
    check("dense_ax", np.max(np.abs(P.ax(Q @ ug) - ref)) < 1e-12 * np.max(np.abs(ref)))
    _, inv = np.unique(m.gid, return_inverse=True)
    ref_minv = np.where(m.mask > 0, 1.0 / np.diag(K)[inv], 0.0)
    check("dense_jacobi", np.allclose(P.minv(), ref_minv, rtol=1e-12))
    check("mult", np.array_equal(P.gs(np.ones(m.n_local), mask=False), P.mult()))
    # Helmholtz: dense K + Q^T diag(h2 B) Q and its diagonal
    x_, y_, z_ = m.xyz()
    h2 = 2.0 + np.cos(3.0 * x_) * np.sin(2.0 * y_) + z_
    P.set_h2(h2)
    Hm = K + Q.T @ np.diag(h2 * Bm.reshape(-1)) @ Q
    refh = Q @ (mask_g * (Hm @ ug))
    check("dense_helmholtz_ax", np.max(np.abs(P.ax(Q @ ug) - refh)) < 1e-12 * np.max(np.abs(refh)))
    check("dense_helmholtz_jacobi", np.allclose(P.minv(), np.where(m.mask > 0, 1.0 / np.diag(Hm)[inv], 0.0),
                                                rtol=1e-12))
    P.set_h2(None)
    # volume of a smoothly deformed cube (GLL quadrature of J is exact there)
    ms = W.box_mesh(3, 2, 2, 3, amp=0.1)
    Ps = oracle.Problem(ms)
    _, B = Ps.geom()
    check("volume", abs(Ps.dot(np.ones(ms.n_local), Ps.gs(B, mask=False)) - 1.0) < 1e-13)
    # PCG vs dense solve, with the iteration bound
    b = W.random_global_rhs(m, 1)
    x, info = P.pcg(b, tol=1e-13, max_iter=400)
    _, first = np.unique(m.gid, return_index=True)
    F = mask_g > 0
    xg = np.zeros(K.shape[0])
    xg[F] = np.linalg.solve(K[np.ix_(F, F)], b[first][F])
    xd = Q @ xg
    check("pcg_dense", info["status"] == 0 and np.linalg.norm(x - xd) < 1e-10 * np.linalg.norm(xd)
          and info["iters"] <= 2 * int(F.sum()))
    # refinement with the inner direction kept: one continued CG, about the
    # FP64 PCG iteration count (bounded so that a broken variant ends quickly)
    mc, h1c, bc = W.deformed_cube(4, 7, seed=2)
    Pc = oracle.Problem(mc, h1c)
    _, i64 = Pc.pcg(bc, tol=1e-10, max_iter=1000)
    _, ic = Pc.ir(bc, tol=1e-10, inner_tol=1e-2, carry=True, max_outer=8, max_inner=400)
    check("ir_kept_direction", ic["status"] == 0 and ic["relres"] <= 1e-10
          and ic["inner"] <= 1.05 * i64["iters"])
    return failed


@pytest.fixture(scope="module")
def builddir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def _build(src_text: str, path: str):
    c = path + ".c"
    with open(c, "w") as fh:
        fh.write(src_text)
    inc = os.path.dirname(SRC)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-I", inc,
                    c, "-o", path + ".so", "-lm"], check=True)
    return oracle.configure(ctypes.CDLL(path + ".so"))


def _with_lib(lib, fn):
    saved = oracle._lib
    oracle._lib = lib
    try:
        return fn()
    finally:
        oracle._lib = saved


def test_battery_passes_on_oracle(builddir):
    lib = _build(open(SRC).read(), str(builddir / "clean"))
    assert _with_lib(lib, _battery) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_battery_catches_mutant(name, builddir):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if name == "h1_at_wrong_point_in_jacobi":
        # the point's own index, as if h1 were taken at (i,j,k) inside the sum
        src = src.replace("const int64_t La = o + k * lx * lx + j * lx + l;",
                          "const int64_t La = o + k * lx * lx + j * lx + l;\n"
                          "                        const int64_t L0 = o + k * lx * lx + j * lx + i;")
    # the FP64 routines come first in the source; the FP32 inner-solve copies later
    assert src.count(old) >= 1, name
    lib = _build(src.replace(old, new, 1), str(builddir / name))
    failed = _with_lib(lib, _battery)
    assert failed, f"mutant {name} passed every pin"
