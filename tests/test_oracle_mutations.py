"""The pins have teeth: plant one plausible mistake at a time in a temporary
copy of the oracle's C source (never in the committed file, always on the
CPU), build it, and require that at least one pin rejects the result."""
import os

import pytest

import oracle
import test_oracle_adjoint as AD
import test_oracle_bruteforce as BF
import test_oracle_cpml as CP
import test_oracle_dynamics as DY
import test_oracle_free_surface as FS
import test_oracle_stencil as ST
import test_oracle_vd as VD


def _dense(orc):
    BF.test_dense_stepper_agrees(orc, (11, 10, 12), 2, 8)
    BF.test_dense_stepper_agrees(orc, (9, 12, 10), 3, 6)


def _poly(orc):
    ST.test_laplacian_exact_on_polynomials(orc, 8)


def _coeffs(orc):
    ST.test_coeffs_match_textbook_closed_form(orc, 8)


def _energy(orc):
    DY.test_energy_conserved_without_damping(orc)
    DY.test_energy_decrement_with_damping_is_exact(orc)


def _reciprocity(orc):
    BF.test_reciprocity_heterogeneous_damped(orc)


def _standing(orc):
    DY.test_standing_wave_is_exact(orc, 8)


def _adjoint(orc):
    AD.test_dot_product(orc)
    AD.test_adjoint_is_the_explicit_transpose(orc)


def _fs(orc):
    FS.test_odd_image_laplacian_is_exact_at_the_surface(orc)
    FS.test_dense_stepper_with_free_surface(orc, (11, 10, 12), 2)
    FS.test_adjoint_dot_product_with_free_surface(orc)


def _cpml(orc):
    CP.test_dense_stepper_agrees(orc, (12, 10, 11), 3, False)


def _vd_dense(orc):
    for cpml in (False, True):
        VD.test_dense_stepper_agrees(orc, (11, 10, 12), 2, cpml)


def _vd_poly(orc):
    VD.test_dplus_exact_on_polynomials(orc)
    VD.test_dminus_exact_on_polynomials(orc)


def _vd_coeffs(orc):
    VD.test_staggered_coeffs_closed_form(orc, 8)


def _vd_energy(orc):
    VD.test_energy_conserved_without_layers(orc)
    VD.test_energy_change_with_damping_is_exact(orc)


def _vd_standing(orc):
    VD.test_standing_wave_is_exact(orc)


def _vd_fs(orc):
    VD.test_standing_wave_with_free_surface_is_exact(orc)
    VD.test_energy_conserved_with_free_surface(orc)
    VD.test_dense_stepper_with_free_surface(orc, (11, 10, 12), 2, False)


def _grad(orc):
    for kind in ("point", "smooth", "source"):
        AD.test_gradient_matches_finite_differences(orc, kind)


MUTATIONS = [
    ("damping drops (1 - eta dt) on u^{n-1}", "(1.0 - e) * up[o]", "up[o]", [_energy, _dense]),
    ("damping sign flipped", "un[o] = (2.0 * ucur[o] - (1.0 - e) * up[o] + C[o] * L) / (1.0 + e);",
     "un[o] = (2.0 * ucur[o] - (1.0 - e) * up[o] + C[o] * L) / (1.0 - e);", [_energy, _dense]),
    ("y axis uses the x weights", "ly += cy[m]", "ly += cx[m]", [_poly, _dense]),
    ("z neighbour uses the y stride", "u[o - m * g->sz]", "u[o - m * g->sy]", [_poly, _dense, _energy]),
    ("centre term dropped on x", "lx += cx[m] * (u[o + m] + u[o - m] - 2.0 * p)",
     "lx += cx[m] * (u[o + m] + u[o - m] - p)", [_poly, _standing]),
    ("Taylor right-hand side wrong", "(p == 1) ? 1.0 : 0.0", "(p == 1) ? 2.0 : 0.0", [_coeffs, _poly]),
    ("source outside the (1 + eta dt) division", "(cell * (1.0 + e))", "cell", [_dense, _reciprocity]),
    ("source sign flipped", "un[o] += C[o] * (double)wavelet[(long)s * nt + n] / (cell * (1.0 + e));",
     "un[o] -= C[o] * (double)wavelet[(long)s * nt + n] / (cell * (1.0 + e));", [_dense]),
    ("receivers record u^n instead of u^{n+1}", "traces[(long)n * nrec + r] = un[", "traces[(long)n * nrec + r] = ucur[",
     [_dense]),
    ("damping profile shifted by one cell", "if (nbl - i > d) d = nbl - i;", "if (nbl - i - 1 > d) d = nbl - i - 1;",
     [_dense]),
    ("leapfrog uses 2 u^{n-1}", "un[o] = 2.0 * ucur[o] - up[o] + C[o] * L;",
     "un[o] = 2.0 * ucur[o] - 2.0 * up[o] + C[o] * L;", [_standing, _dense]),
    ("adjoint applies C after L (the forward's order)", "cm[o] = C[o] * m1[o];", "cm[o] = m1[o] * (1.0 + 0.0 * C[o]);",
     [_adjoint]),
    ("adjoint residual outside the damping division", "m0[o] += resid[(long)(n - 1) * nrec + r] / (1.0 + e);",
     "m0[o] += resid[(long)(n - 1) * nrec + r];", [_adjoint]),
    ("adjoint source misses the 1/h^3 cell factor", "if (adj) adj[(long)s * nt + (n - 1)] = C[o] * m0[o] / cell;",
     "if (adj) adj[(long)s * nt + (n - 1)] = C[o] * m0[o];", [_adjoint]),
    ("gradient drops its source term", "+= m0[o] * (double)wavelet[(long)s * nt + (n - 1)] / cell;",
     "+= 0.0 * m0[o] * (double)wavelet[(long)s * nt + (n - 1)] / cell;", [_grad]),
    ("gradient pairs mu^n with u^n", "const double *u = u_hist[n];   /* u^{n-1} */",
     "const double *u = u_hist[n + 1];", [_grad]),
    ("free surface uses the even image", "u[at(g, i, j, -m)] = -u[at(g, i, j, m)];",
     "u[at(g, i, j, -m)] = u[at(g, i, j, m)];", [_fs]),
    ("free surface keeps the top damping layer", "for (int k = 0; k < nbl && k < nz - 1 - nbl; ++k) ez[k] = 0.0;\n    for (int k = 0; k < nz; ++k)\n        for (int j = 0; j < ny; ++j)\n            for (int i = 0; i < nx; ++i) {\n                const long q",
     "for (int k = 0; k < 0; ++k) ez[k] = 0.0;\n    for (int k = 0; k < nz; ++k)\n        for (int j = 0; j < ny; ++j)\n            for (int i = 0; i < nx; ++i) {\n                const long q", [_fs]),
    ("adjoint misses the surface projection", "if (free_surface) zero_top(&g, m0);", "", [_fs]),
    ("CPML memory forgets its decay", "psi[a][o] = B[a][idx[a]] * psi[a][o] + gg * d1 / hh[a];",
     "psi[a][o] = psi[a][o] + gg * d1 / hh[a];", [_cpml]),
    ("CPML drops the second memory variable", "total += d2 + dpsi + zeta[a][o];", "total += d2 + dpsi;", [_cpml]),
    ("staggered D- offsets swapped", "dv += aw[m] * (v[a][o + (m - 1) * stride[a]] - v[a][o - m * stride[a]]);",
     "dv += aw[m] * (v[a][o + m * stride[a]] - v[a][o - (m - 1) * stride[a]]);", [_vd_poly, _vd_energy]),
    ("staggered weights: wrong consistency right-hand side", "A[q][R] = (q == 0) ? 0.5 : 0.0;",
     "A[q][R] = (q == 0) ? 1.0 : 0.0;", [_vd_coeffs, _vd_poly]),
    ("half-point buoyancy not averaged", "? 0.5 * (Bc[o] + Bc[o + stride[a]]) : Bc[o];", "? Bc[o] : Bc[o];",
     [_vd_dense]),
    ("K = rho v instead of rho v^2", "K[o] = rr * vv * vv;", "K[o] = rr * vv;", [_vd_standing, _vd_dense]),
    ("velocity damping at grid-point positions", "eta += prof[c][c == a][0][idx[c]];", "eta += prof[c][0][0][idx[c]];",
     [_vd_dense, _vd_energy]),
    ("VD source outside the (1 + e/2) division", "(double)wavelet[(long)s * nt + n] / (cell * (1.0 + 0.5 * e));",
     "(double)wavelet[(long)s * nt + n] / cell;", [_vd_dense]),
    ("VD CPML drops the pressure-gradient memory", "dp += psi[a][o];", "dp += 0.0 * psi[a][o];", [_vd_dense]),
    ("VD surface: v_z mirrored odd", "vz[at(g, i, j, -m)] = vz[at(g, i, j, m - 1)];",
     "vz[at(g, i, j, -m)] = -vz[at(g, i, j, m - 1)];", [_vd_fs]),
    ("VD surface: v_z mirrored without the half-cell shift", "vz[at(g, i, j, -m)] = vz[at(g, i, j, m - 1)];",
     "vz[at(g, i, j, -m)] = vz[at(g, i, j, m)];", [_vd_fs]),
    ("VD surface: p mirrored even", "p[at(g, i, j, -m)] = -p[at(g, i, j, m)];",
     "p[at(g, i, j, -m)] = p[at(g, i, j, m)];", [_vd_fs]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pins):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mut_src = tmp_path / "oracle_mut.c"
    mut_src.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mut_src), out=str(tmp_path / "liboracle_mut.so"))
    orc = oracle.Oracle(lib)
    failures = []
    for pin in pins:
        try:
            pin(orc)
        except (AssertionError, ValueError) as e:  # the pin rejected the mutant
            failures.append(f"{pin.__name__}: {type(e).__name__}")
    assert failures, f"no pin caught: {name}"
    assert os.path.exists(lib)
