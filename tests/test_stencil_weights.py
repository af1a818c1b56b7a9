"""The library's optimised stencil weights (host code, no GPU) against the
oracle's (reading R16): two independent solvers of the same constrained
least-squares problem (KKT elimination with trapezoid quadrature in the
oracle; null-space Cholesky with Simpson quadrature in the library) must
agree to the quadrature error."""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M


@pytest.mark.parametrize("kmax", [np.pi / 2, 2 * np.pi / 3, 0.9 * np.pi])
def test_library_weights_match_oracle(orc, kmax):
    c_lib = M.mmod_optimized_coefficients(kmax)
    c_orc = orc.optimized_coeffs(8, kmax, nq=20000)[1:]
    assert np.max(np.abs(c_lib - c_orc)) < 1e-7, (c_lib, c_orc)
    assert abs(np.dot([1, 4, 9, 16], c_lib) - 1.0) < 1e-12


def test_library_rejects_bad_band():
    lib = M.load()
    out = np.zeros(4)
    for bad in (0.0, -1.0, 4.0):
        assert lib.mmod_optimized_coefficients(bad, out.ctypes.data) == -1
