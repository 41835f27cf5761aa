"""Failure paths through the C ABI, without faulting or hanging the GPU.

  * A bounded device wait that runs out (an mbarrier that nothing arrives on, waited on
    with the library's bounded wait) is counted on the device, read back by the host and
    returned as MX_ETIMEOUT; the handle and the context stay usable and the next solve is
    correct.
  * Pivot growth of the no-pivot local LU (coercivity, Lemma 2.2, keeps pivots nonzero,
    Sec. 3.3, but does not bound their growth): mx_info reports max|U| / max|A^l|, which
    must equal the growth of a dense no-pivot LU of the oracle's minors; a limit below it
    makes mx_factor return MX_ESINGULAR and leaves the handle unfactored."""
import time

import pytest

import inputs
from oracle.problem import Problem as OracleProblem
from parity import assert_close, nopivot_growth

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounded_wait_times_out_and_the_handle_stays_usable():
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(1, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, _ = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with mx.Problem(n, k, k, k, 5, 1, 5, mx.MX_MIXED) as P:
        P.factor()
        t0 = time.perf_counter()
        rc = mx.mx_test_bounded_wait(P.h, 1024, 4)
        dt = time.perf_counter() - t0
        assert rc == mx.MX_ETIMEOUT, rc
        assert "4 bounded waits ran out" in mx.mx_last_error()
        assert dt < 30.0, dt
        for bad in ((0, 4), (1024, 0)):
            assert mx.mx_test_bounded_wait(P.h, *bad) == mx.MX_EINVAL
        # the same handle and context afterwards: a solve zeroes the word at its start
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK and all(s["converged"] for s in st)
    assert_close(x, xo.T, 1e-8, what="solve after a timed-out wait")


@pytest.mark.parametrize("prec,bc", [(mx.MX_MIXED, mx.MX_BC_PEC), (mx.MX_PLAIN_FP64, mx.MX_BC_PEC),
                                     (mx.MX_MIXED, mx.MX_BC_IMPEDANCE)])
def test_reported_growth_equals_the_oracle_minors_growth(prec, bc):
    n, k, xi, core = 6, 4.0, 4.0, 3
    imp = bc == mx.MX_BC_IMPEDANCE
    O = OracleProblem(n, k, xi, xi, core, 1, bc="imp" if imp else "pec")
    g = [nopivot_growth(O.dd.minor(l).toarray()) for l in range(len(O.dd.idx))]
    with mx.Problem(n, k, xi, xi, core, 1, 0, prec, bc=bc) as P:
        assert mx.mx_info(P.h)["growth_subdomain"] == -1
        P.factor()
        info = mx.mx_info(P.h)
    # the device takes moduli in FP32 (and the mixed form factors in c64)
    tol = 2e-4 if prec == mx.MX_MIXED else 1e-6
    print("growth", info["max_growth"], "oracle", max(g), "subdomain", info["growth_subdomain"])
    assert abs(info["max_growth"] - max(g)) <= tol * max(g), (info["max_growth"], max(g))
    l = info["growth_subdomain"]
    assert 0 <= l < len(g) and abs(g[l] - max(g)) <= tol * max(g)


def test_growth_over_the_limit_returns_esingular_and_leaves_the_handle_unfactored():
    n, k = 6, 4.0
    c, p = inputs.bump_batch(2, 1)
    with mx.Problem(n, k, k, k, 3, 1, 0, mx.MX_MIXED) as P:
        P.factor()
        g = mx.mx_info(P.h)["max_growth"]
        assert 0 < g < 1e6  # far below the default limit of the c64 factors
        mx.mx_set_growth_limit(P.h, 0.5 * g)
        with pytest.raises(mx.MxError) as e:
            P.factor()
        assert e.value.code == mx.MX_ESINGULAR and "pivot growth" in str(e.value)
        f = P.load_vector(c, p, 0.1)
        with pytest.raises(mx.MxError) as e:
            P.solve(f, tol=1e-8)
        assert e.value.code == mx.MX_ENOTFACTORED
        with pytest.raises(mx.MxError) as e:
            mx.mx_set_growth_limit(P.h, float("nan"))
        assert e.value.code == mx.MX_EINVAL
        mx.mx_set_growth_limit(P.h, 0)  # the default again
        P.factor()
        x, st, rc = P.solve(f, tol=1e-8, restart=0, max_it=200)
    assert rc == mx.MX_OK and st[0]["converged"]
