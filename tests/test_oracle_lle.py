"""Pins of the Lugiato-Lefever form (oracle/lle.py) against the coupled mode equations: Sec. 2
states that the CMEs are a discrete Fourier expansion of a driven and damped NLS (LLE)
equation.  Classic RK4 is covariant under a fixed linear change of variables, so RK4 on the
LLE in the time domain and RK4 on the CMEs (the oracle's direct O(N^3) sum) must give the same
field to round-off once the mode amplitudes are transformed to theta_j.  Also the LLE's
homogeneous stationary state, a closed form.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import lle
from paper_1307_3428_gb300 import workloads as wl


@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("alpha,beta,F", [(0.0, -0.0125, 1.7), (2.5, 0.04, 2.0 + 0.5j),
                                          (-1.0, -0.3, 0.8)])
def test_lle_rk4_is_the_cme_rk4_in_the_fourier_basis(N, alpha, beta, F):
    inst = wl.lle_instance(N, alpha, beta, F, noise=0.3, seed=40 + N)
    h, n = 2e-3, 60
    cme = oracle.integrate(inst, h, n, oracle.RK4)
    psi = lle.rk4(lle.modes_to_theta(inst.D0), alpha, beta, F, h, n)
    assert np.max(np.abs(lle.theta_to_modes(psi) - cme)) <= 1e-12 * np.max(np.abs(cme))


def test_lle_homogeneous_stationary_state():
    """psi constant with F = psi (1 + i (alpha - |psi|^2)): the cubic
    P (1 + (alpha - P)^2) = |F|^2, which is the CW cubic of the CMEs with kappa_0 = 2,
    kappa_ext = g0 = 1 and sigma = alpha."""
    alpha, F = 3.0, 2.2
    for P in cf.cw_powers(alpha, F, 2.0, 1.0, 1.0):
        psi0 = cf.cw_field(P, alpha, F, 2.0, 1.0, 1.0)
        psi = np.full(16, psi0, dtype=complex)
        assert np.max(np.abs(lle.rhs(psi, alpha, -0.02, F))) <= 1e-12 * abs(F)
