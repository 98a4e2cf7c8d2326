"""The Lugiato-Lefever form on the GPU: an LLE instance (workloads.lle_instance) stepped by the
library's RK4IP and Strang kernels, with the time-domain field psi(theta_j) read through
cme_transform (+1), against classic RK4 on the LLE in the time domain (oracle/lle.py, itself
pinned to the CME oracle).  The reference takes an eighth of the step: plain RK4 on the stiff
dispersion term (h |beta/2| mu^2 up to 0.33 at N = 256) would otherwise be the least accurate
of the three.  RK4IP then agrees to 1e-7 and Strang (second order) to 2e-5."""
import numpy as np
import pytest

from oracle import lle
from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    cme.load()


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


CASES = [(0.0, -0.0125, 1.2 * np.sqrt(2.0)), (2.5, -0.04, 2.0), (4.0, 0.02, 1.6 + 0.3j)]


@pytest.mark.parametrize("integ,tol", [(cme.RK4IP, 1e-7), (cme.STRANG, 2e-5)])
@pytest.mark.parametrize("N", [64, 256])
def test_time_domain_field_matches_the_lle(N, integ, tol):
    insts = [wl.lle_instance(N, a, b, F, noise=1e-2, seed=5000 + k)
             for k, (a, b, F) in enumerate(CASES)]
    h, n = 1e-3, 400
    bt = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=cme.FP64,
                   integrator=integ)
    bt.step(h, n)
    psi_gpu = bt.split(bt.transform(+1))
    for inst, (a, b, F), got in zip(insts, CASES, psi_gpu):
        ref = lle.rk4(lle.modes_to_theta(inst.D0), a, b, F, h / 8, 8 * n)
        assert rel(got, ref) <= tol, (a, b, F, rel(got, ref))
