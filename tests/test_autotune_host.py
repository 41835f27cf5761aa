"""Host logic of the autotuner on CPU, with stand-ins for the device measurements: which
knobs apply to which problem, the coordinate search (planted optimum, noise threshold,
non-converging settings), the measurement sequence against a fake problem, and the JSON
cache (hit without measuring, unreadable files, foreign entries)."""
import json

import pytest

at = pytest.importorskip("paper_1711_03789_gb300.autotune")
mx = pytest.importorskip("paper_1711_03789_gb300")


def _info(prec, n_coarse=0):
    return {"precision": prec, "n_coarse": n_coarse, "n_dof": 1000, "n_sub": 8, "max_local": 200,
            "coarse_band": 40 if n_coarse else 0}


def _applicable(info, cfg=None):
    cfg = dict(at.DEFAULTS, **(cfg or {}))
    return {k for k in at.KNOBS if at.candidates(info, cfg, k)}


def test_candidates_per_problem_kind():
    assert _applicable(_info(mx.MX_PLAIN_FP64)) == {"local_rhs_group"}
    assert _applicable(_info(mx.MX_PLAIN_FP64, 125)) == {"local_rhs_group", "coarse_blocks"}
    assert _applicable(_info(mx.MX_MIXED)) == {"lu_tensor", "dots", "local_tensor", "local_rhs_group"}
    mixed_coarse = _info(mx.MX_MIXED, 125)
    assert _applicable(mixed_coarse) == {"lu_tensor", "dots", "coarse_inverse", "local_tensor", "local_rhs_group"}
    # the cooperative sweep only runs when the explicit inverse is off
    assert "coarse_blocks" in _applicable(mixed_coarse, {"coarse_inverse": 0})
    # the persistent LU's grid: only for the persistent LU and more subdomains than SMs
    many = dict(mixed_coarse, n_sub=1728)
    assert "lu_grid" in _applicable(many) and "lu_grid" not in _applicable(many, {"lu_tensor": 4})
    assert at.candidates(many, at.DEFAULTS, "lu_grid")[0] == 0
    # the single-TF32 LU update changes the factors' accuracy: only on request
    assert 1 not in at.candidates(mixed_coarse, at.DEFAULTS, "lu_tensor")
    assert 1 in at.candidates(mixed_coarse, at.DEFAULTS, "lu_tensor", allow_reduced=True)
    for name in at.KNOBS:
        for v in at.candidates(mixed_coarse, dict(at.DEFAULTS, coarse_inverse=0), name, True):
            assert at.DEFAULTS[name] in at.candidates(mixed_coarse, dict(at.DEFAULTS, coarse_inverse=0), name, True)
            assert isinstance(v, int)


def _separable(target, weights):
    """Cost with its minimum at `target`: each knob away from its target adds its weight."""
    calls = []

    def measure(knobs):
        calls.append(dict(knobs))
        return 100.0 + sum(w for k, w in weights.items() if knobs[k] != target[k]), {"converged": True}

    return measure, calls


def test_search_finds_a_planted_optimum():
    info = _info(mx.MX_MIXED, 125)
    target = dict(at.DEFAULTS, lu_tensor=3, dots=1, coarse_inverse=0, local_tensor=0, local_rhs_group=4,
                  coarse_blocks=38)
    measure, calls = _separable(target, {k: 10.0 for k in at.KNOBS})
    knobs, cost, base, trials = at.search(info, measure)
    assert knobs == target and cost == 100.0
    assert base == 100.0 + 10.0 * 6
    # one trial per value: the default, then every other candidate of each knob once
    cfg = dict(at.DEFAULTS)
    expect = 1
    for name in at.KNOBS:
        expect += len([v for v in at.candidates(info, cfg, name) if v != cfg[name]])
        cfg[name] = target[name]
    assert len(calls) == len(trials) == expect
    assert len({tuple(sorted(c.items())) for c in calls}) == len(calls)


def test_search_keeps_defaults_within_noise():
    info = _info(mx.MX_MIXED)

    def measure(knobs):  # every other setting 1 % faster: below the 2 % threshold
        return (100.0 if knobs == at.DEFAULTS else 99.0), {"converged": True}

    knobs, cost, base, _ = at.search(info, measure, min_gain=0.02)
    assert knobs == at.DEFAULTS and cost == base == 100.0
    knobs, _, _, _ = at.search(info, measure, min_gain=0.0)
    assert knobs != at.DEFAULTS


def test_search_never_picks_a_setting_that_does_not_converge():
    info = _info(mx.MX_MIXED)

    def measure(knobs):
        if knobs["lu_tensor"] == 3:
            return float("inf"), {"converged": False}
        return (50.0 if knobs["local_tensor"] == 0 else 100.0), {"converged": True}

    knobs, cost, _, trials = at.search(info, measure)
    assert knobs["lu_tensor"] == 0 and knobs["local_tensor"] == 0 and cost == 50.0
    assert any(not t["converged"] for t in trials)
    with pytest.raises(RuntimeError):
        at.search(info, lambda k: (float("inf"), {"converged": False}))


class FakeProblem:
    """Stand-in for Problem: records knob settings, factorisations and solves; the device
    times depend on the knobs as a planted cost model."""

    def __init__(self, prec=mx.MX_MIXED, n_coarse=125, converge=lambda knobs: True):
        self._info = _info(prec, n_coarse)
        self.knobs = {}
        self.log = []
        self.converge = converge
        self.factored_with = None

    def info(self):
        return dict(self._info)

    def set_tuning(self, key, value):
        name = {v: k for k, v in at.KNOBS.items()}[key]
        self.knobs[name] = value
        self.log.append(("set", name, value))

    def factor(self):
        self.factored_with = dict(self.knobs)
        self.log.append(("factor",))

    def solve(self, rhs, tol, restart, max_it, x=None):
        self.log.append(("solve", tol, restart, max_it))
        ok = self.converge(self.knobs)
        st = [dict(iterations=20, converged=ok, rel_residual=tol / 2, rel_estimate=tol / 2) for _ in range(2)]
        return rhs, st, mx.MX_OK if ok else mx.MX_ENOCONV

    def timings(self):
        k = self.factored_with or {}
        factor_ms = 50.0 - (20.0 if k.get("lu_tensor") == 3 else 0.0)
        solve_ms = 30.0 - (5.0 if self.knobs.get("local_rhs_group") == 8 else 0.0)
        return {"factor_ms": factor_ms, "solve_ms": solve_ms}


def test_measure_sequence_against_a_fake_problem():
    P = FakeProblem()
    m = at.make_measure(P, rhs="b", tol=1e-6, max_it=77, repeats=2, solves_per_factor=3.0)
    cost, det = m(dict(at.DEFAULTS, lu_tensor=3))
    assert cost == pytest.approx(30.0 + 3.0 * 30.0)
    assert det == {"factor_ms": 30.0, "solve_ms": 30.0, "iterations": 20, "converged": True}
    # every knob set before the factorisation, then one warm-up and two timed solves
    kinds = [e[0] for e in P.log]
    assert kinds == ["set"] * len(at.KNOBS) + ["factor", "solve", "solve", "solve"]
    assert all(e[1:] == (1e-6, 0, 77) for e in P.log if e[0] == "solve")
    P2 = FakeProblem(converge=lambda knobs: knobs.get("local_tensor") != 0)
    cost, det = at.make_measure(P2, rhs="b")(dict(at.DEFAULTS, local_tensor=0))
    assert cost == float("inf") and not det["converged"]


def test_tune_applies_caches_and_reuses(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    P = FakeProblem()
    out = at.tune(P, nrhs=2, cache_path=path, device="GB300-test", rhs="b", repeats=1)
    assert not out["cached"]
    assert out["knobs"]["lu_tensor"] == 3 and out["knobs"]["local_rhs_group"] == 8
    assert out["cost_ms"] == pytest.approx(30.0 + 25.0) and out["default_ms"] == pytest.approx(80.0)
    # left factored under the chosen knobs
    assert P.log[-1] == ("factor",) and P.factored_with == out["knobs"]
    data = json.load(open(path))
    assert data["format"] == at.FORMAT and len(data["entries"]) == 1
    key = at.cache_key(P.info(), 2, "GB300-test")
    assert data["entries"][key]["knobs"] == out["knobs"]

    # same shape, device and batch: applied without measuring
    P2 = FakeProblem()

    def fail(knobs):
        raise AssertionError("measured on a cache hit")

    out2 = at.tune(P2, nrhs=2, cache_path=path, device="GB300-test", measure=fail)
    assert out2["cached"] and out2["knobs"] == out["knobs"] and P2.factored_with == out["knobs"]
    # another batch size or device is another key
    assert at.cache_key(P.info(), 4, "GB300-test") != key
    assert at.cache_key(P.info(), 2, "other") != key
    assert at.cache_key(P.info(), 2, "GB300-test", tag="hras") != key
    out3 = at.tune(FakeProblem(), nrhs=4, cache_path=path, device="GB300-test", rhs="b", repeats=1)
    assert not out3["cached"]
    assert len(json.load(open(path))["entries"]) == 2


@pytest.mark.parametrize("text", ["", "{not json", "[1, 2]", '{"format": 99, "entries": {}}'])
def test_unreadable_cache_reads_as_empty(tmp_path, text):
    path = tmp_path / "tune.json"
    path.write_text(text)
    assert at.Cache(str(path)).entries == {}
    out = at.tune(FakeProblem(), nrhs=2, cache_path=str(path), device="d", rhs="b", repeats=1)
    assert not out["cached"]
    assert json.load(open(path))["format"] == at.FORMAT


def test_foreign_cache_entries_are_ignored(tmp_path):
    P = FakeProblem()
    key = at.cache_key(P.info(), 2, "d")
    path = tmp_path / "tune.json"
    bad = {"knobs": {"no_such_knob": 1}}
    path.write_text(json.dumps({"format": at.FORMAT, "entries": {key: bad}}))
    assert at.Cache(str(path)).get(key) is None
    out = at.tune(P, nrhs=2, cache_path=str(path), device="d", rhs="b", repeats=1)
    assert not out["cached"] and "no_such_knob" not in P.knobs
