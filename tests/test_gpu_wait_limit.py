"""Failure handling of the bounded device-side waits, without a GPU fault.

Every grid exchange and barrier of the persistent Krylov kernels gives up
after a bounded number of clock cycles, records a timeout and leaves; the
call returns RBFFD_ETIMEOUT.  The bound is settable per context, so this
test makes the waits run out (a limit of two cycles: no exchange across
many CTAs completes that fast), checks the status, and then checks that the
same context and problem still solve correctly once the default is back.
Nothing hangs: every block leaves at its next wait."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_l2
from paper_2106_07616_gb300 import _build, clouds, rbffd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", [rbffd.PRECOND_JACOBI, rbffd.PRECOND_AMG_FGMRES])
def test_wait_limit_times_out_and_the_context_recovers(precond):
    _build.build()
    fp = clouds.cavity(100, dt=0.1)  # 10 000 rows: every solve spans many CTAs
    c = rbffd.Context(0)
    P = rbffd.Problem(c, fp, precond=precond)
    c.set_wait_limit(1)
    with pytest.raises(rbffd.RbffdError) as e:
        P.simple_iterate(fp.dt, krylov_tol=1e-12, krylov_maxit=100000)
    assert e.value.code == rbffd.ETIMEOUT, e.value
    c.set_wait_limit(0)
    P.reload(fp, precond=precond)  # the timed-out iteration left its fields unspecified
    O = oracle.Problem(fp, krylov_tol=1e-12, krylov_maxit=100000)
    dg, sg = P.simple_iterate(fp.dt, krylov_tol=1e-12, krylov_maxit=100000)
    do, so = O.simple_iterate(fp.dt)
    assert abs(dg - do) <= 1e-8 * abs(do), (dg, do)
    for k in ("u", "v", "p"):
        assert rel_l2(P.get(k), O.get(k)) <= 1e-8, k
    P.close()
    c.close()


def test_wait_limit_range():
    c = rbffd.Context(0)
    for bad in (-1, 41):
        with pytest.raises(rbffd.RbffdError) as e:
            c.set_wait_limit(bad)
        assert e.value.code == rbffd.EINVAL
    c.set_wait_limit(40)
    c.set_wait_limit(0)
    c.close()
