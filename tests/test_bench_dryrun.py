"""bench.py's main paths on CPU with stand-ins for the library and for CUDA: the default
solve benchmark (JSON contract keys, roofline, per-kernel table, e2e byte counts, launch
count), the autotuner path (search, then a cache hit) and the serving mix with an offered-load
sweep, and the oracle arm (rank 0 prints, other ranks exit). Nothing here measures anything;
it checks that the host code runs end to end and emits the line the contract asks for."""
import contextlib
import io
import json
import sys
import types

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from paper_1711_03789_gb300 import _lib as L  # noqa: E402
from paper_1711_03789_gb300 import autotune as real_autotune  # noqa: E402

N_DOF = 1000


class FakeProblem:
    log = []

    def __init__(self, n, k, xp, xq, core, ov, cm, prec, stream=None, dense_local=False, bc=0):
        FakeProblem.log.append(("Problem", n, k, xp, xq, core, ov, cm, prec, bc))
        self.h, self.n_dof = 1, N_DOF

    def set_tuning(self, key, v):
        FakeProblem.log.append(("tune", key, v))

    def set_coarse_solver(self, *a):
        FakeProblem.log.append(("coarse", a))

    def factor(self):
        FakeProblem.log.append(("factor",))

    def load_vector(self, c, p, w, out=None):
        FakeProblem.log.append(("load", tuple(out.shape)))
        return out

    def solve(self, f, tol, restart, max_it, x=None):
        FakeProblem.log.append(("solve", tol, restart, max_it))
        st = [dict(iterations=35, converged=True, rel_residual=9e-7, rel_estimate=9e-7)] * f.shape[0]
        return x, st, 0

    def timings(self):
        return dict(build_ms=1.0, factor_ms=2.0, solve_ms=3.0, solve_launches=10, restarts=0, max_iterations=35,
                    coarse_inner_iterations=0, coarse_inner_solves=0)

    def info(self):
        return dict(n_dof=N_DOF, nnz=1, n_sub=8, max_local=10, sum_local=80, n_coarse=27, nnz_r0=1, factor_bytes=1,
                    coarse_band=3, precision=1)

    def close(self):
        pass


class FakeEvent:
    def __init__(self, **kw):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 600.0


@pytest.fixture
def fakes(monkeypatch):
    fake = types.ModuleType("paper_1711_03789_gb300")
    for name in dir(L):
        if name.startswith("MX_"):
            setattr(fake, name, getattr(L, name))
    fake.Problem = FakeProblem
    fake.autotune = real_autotune
    fake.use_torch_allocator = lambda dev: None
    fake.mx_set_tuning = lambda h, key, v: FakeProblem.log.append(("tune", key, v))
    fake.mx_set_weighted_gmres = lambda h, v: None
    fake.mx_set_preconditioner = lambda h, v: None
    fake.mx_profile = lambda on: None
    count = [0]

    def launch_count():
        count[0] += 100
        return count[0]

    fake.mx_launch_count = launch_count
    fake.mx_profile_read = lambda: {
        "local_solve": dict(ms=10.0, launches=70, bytes=70 * 16e9, flops=70 * 1e9),
        "spmv": dict(ms=2.0, launches=70, bytes=70 * 1e9, flops=70 * 1e8),
        "unused": dict(ms=0.0, launches=0, bytes=0.0, flops=0.0)}
    tickets = []
    fake.mx_server_create = lambda budget, workers=2: object()
    fake.mx_server_destroy = lambda s: None

    def submit(s, n, k, xp, xq, c, p, **kw):
        tickets.append(c.shape[0])
        return len(tickets) - 1

    fake.mx_server_submit = submit
    fake.mx_server_poll = lambda s, t, n, nrhs: (None, [dict(converged=True)] * nrhs, dict(latency_ms=10.0 + t), 0)
    fake.mx_server_stats = lambda s: dict(batches=3, factorisations=4, evictions=0, cached_bytes=5 << 30)
    monkeypatch.setitem(sys.modules, "paper_1711_03789_gb300", fake)

    empty = torch.empty

    def cpu_empty(*a, **kw):
        kw.pop("pin_memory", None)
        kw.pop("device", None)
        return empty(*a, **kw)

    monkeypatch.setattr(torch, "empty", cpu_empty)
    monkeypatch.setattr(torch, "empty_like", lambda t: empty(t.shape, dtype=t.dtype))
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda: (100 * 2 ** 30, 200 * 2 ** 30))
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    FakeProblem.log = []
    return fake


def _run(monkeypatch, argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1, lines
    return json.loads(lines[0])


def test_default_solve_benchmark_line(fakes, monkeypatch):
    line = _run(monkeypatch, ["--steps", "2", "--warmup", "3", "--no-cpu-baseline"])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "clocks", "kernels"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] == pytest.approx(0.3) and line["higher_is_better"] is False
    assert line["config"]["workload"] == "maxwell60_k30_2lvl"
    assert line["e2e"]["h2d_bytes_per_step"] == 16 * N_DOF * 16
    assert line["gpu_launches"] == 100
    r = line["roofline"]
    assert r["kernel"] == "local_solve" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert list(line["kernels"]) == ["local_solve", "spmv"]
    # 3 warm-up + 2 timed + 2 end-to-end steps, then one untimed + one timed step of each
    # of the three variant legs; every step: build, factor, load, solve
    problems = [e for e in FakeProblem.log if e[0] == "Problem"]
    assert len(problems) == 13
    assert sum(1 for e in FakeProblem.log if e[0] == "solve") == 13
    # the plain FP64 leg, then xi = k^1.5 on both sides, then the literal xi_prob = 0 setting
    k15 = 30.0 ** 1.5
    assert [e[8] for e in problems[7:9]] == [L.MX_PLAIN_FP64] * 2
    assert [(e[3], e[4]) for e in problems[9:11]] == [(k15, k15)] * 2
    assert [(e[3], e[4]) for e in problems[11:13]] == [(0.0, k15)] * 2
    assert [e[3] for e in FakeProblem.log if e[0] == "solve"][-1] == 400  # max_it of the literal leg
    assert line["plain_fp64"]["value"] == pytest.approx(0.6) and line["mixed_speedup"] == pytest.approx(2.0)
    assert set(line["xi_variants"]) == {"xi_k1.5", "config5_literal"}
    assert line["xi_variants"]["config5_literal"]["max_it"] == 400
    # the bounded serving leg: closed loop and Poisson arrivals at 0.8 x capacity
    sv = line["serving"]
    assert sv["config"]["requests"] == 64 and sv["config"]["restart"] == 30
    assert sv["closed_loop"]["p99_ms"] >= sv["closed_loop"]["p50_ms"] > 0 and "p99_ms" in sv["poisson_0.8x"]


def test_no_variants_runs_only_the_timed_workload(fakes, monkeypatch):
    line = _run(monkeypatch, ["--steps", "2", "--warmup", "3", "--no-cpu-baseline", "--no-variants"])
    assert sum(1 for e in FakeProblem.log if e[0] == "Problem") == 7
    assert "plain_fp64" not in line and "xi_variants" not in line and "serving" not in line


def test_autotune_path_searches_then_hits_the_cache(fakes, monkeypatch, tmp_path):
    cache = str(tmp_path / "tune.json")
    first = _run(monkeypatch, ["--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--autotune", cache])
    assert first["autotune"]["cached"] is False and set(first["autotune"]["knobs"]) == set(real_autotune.KNOBS)
    second = _run(monkeypatch, ["--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--autotune", cache])
    assert second["autotune"]["cached"] is True and second["autotune"]["knobs"] == first["autotune"]["knobs"]


def test_serving_line_with_a_load_sweep(fakes, monkeypatch):
    line = _run(monkeypatch, ["--serving", "--requests", "6", "--loads", "0.5,0.8,1.2", "--budget-gb", "40"])
    assert line["unit"] == "s (p99 latency)"
    assert line["config"]["loads"] == [0.5, 0.8, 1.2] and line["config"]["budget_bytes"] == 40 * 2 ** 30
    for key in ("closed_loop", "poisson_0.5x", "poisson_0.8x", "poisson_1.2x"):
        assert line[key]["converged_rhs"] == line[key]["rhs"], key
        assert line[key]["cached_bytes_at_end"] == 5 << 30, key  # the server's cache when the run ends
    assert line["value"] == pytest.approx(line["poisson_0.8x"]["p99_ms"] / 1e3)


def test_reference_arm_line_and_other_ranks(monkeypatch):
    """The oracle arm on the small 10^3 workload: rank 0 prints the contract line, any other
    rank exits without work."""
    line = _run(monkeypatch, ["--impl", "reference", "--workload", "maxwell10_k6_1lvl", "--steps", "1",
                              "--warmup", "1"])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "maxwell10_k6_1lvl"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    assert buf.getvalue().strip() == ""
