"""The MPdist tolerance rule of the parity tests (tests/tolerance.py), on the
CPU: relative above the floor, the same bound carried into d^2 below it,
continuous at the floor, and below it equivalent to an error of tol / 50 in rho."""
import numpy as np
import pytest

import tolerance


@pytest.mark.parametrize("ell", [4, 32, 256])
def test_rule_is_continuous_at_the_floor_and_scales(ell):
    fl = tolerance.d_floor(ell)
    assert np.isclose(fl, np.sqrt(2 * ell) / 10)              # 1/20 of the largest distance 2 sqrt(ell)
    e = 1e-6
    above = tolerance.profile_errors([fl * (1 + e)], [fl], ell)[0]
    below = tolerance.profile_errors([fl * (1 - 1e-12) * (1 + e)], [fl * (1 - 1e-12)], ell)[0]
    assert np.isclose(above, e) and np.isclose(below, e, rtol=1e-5)
    # exact agreement passes, twice the tolerance fails, above the floor
    tol = 1e-4
    d_ref = np.array([fl, 2 * fl, np.sqrt(ell)])
    assert tolerance.assert_profiles_close(d_ref, d_ref, ell, tol) == 0.0
    with pytest.raises(AssertionError):
        tolerance.assert_profiles_close(d_ref * (1 + 2 * tol), d_ref, ell, tol)


@pytest.mark.parametrize("ell", [8, 64])
def test_below_the_floor_the_rule_is_an_error_in_rho(ell):
    """d = sqrt(2 ell (1 - rho)): an error of tol / 50 in rho is exactly the
    allowance below the floor, whatever d is there (d = 0 included)."""
    tol = 1e-4
    rho_ref = np.array([1.0, 1 - 1e-6, 1 - 1e-3, 0.999])
    d_ref = np.sqrt(2 * ell * (1 - rho_ref))
    assert (d_ref < tolerance.d_floor(ell)).all()
    d = np.sqrt(2 * ell * np.maximum(0.0, 1 - (rho_ref - tol / 50)))
    r = tolerance.profile_errors(d, d_ref, ell)
    assert np.allclose(r, tol)
