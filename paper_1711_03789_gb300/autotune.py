"""Autotuner for the launch-shape and kernel-variant knobs of mx_set_tuning.

For one built problem it times the factorisation plus a preconditioned GMRES solve of a
seeded right-hand-side batch under candidate knob settings and keeps the cheapest setting
whose solves all converge. The search is coordinate-wise (one knob at a time, the others
held at the best values found so far) because each knob steers a different kernel: the LU
trailing update (factor), the coarse inverse (factor and coarse apply), the local solves
(tensor-core or CUDA-core, right-hand-side group) and the cooperative coarse sweep. A
candidate replaces the incumbent only if it is faster by more than `min_gain`, so timing
noise does not flip a knob away from its default.

Choices are cached in a JSON file keyed by the device name, the right-hand-side count, the
problem's shape as mx_info reports it (DOFs, subdomains, largest minor, coarse size and
band, precision) and a caller's tag for what mx_info does not show (wavenumber, shifts,
preconditioner variant, coarse solver), so a later process with the same key applies them
without measuring.

Costs come from mx_timings (CUDA events on the library's stream): cost = factor_ms +
solves_per_factor * solve_ms, the solve time the best of `repeats` solves after one warm-up
solve (the first solve after a factorisation may build the tensor-core panel images).
"""
import json
import os
import tempfile

import numpy as np

from . import _lib as L

# knob name -> mx_set_tuning key; the order is the order of the coordinate search
KNOBS = {
    "lu_tensor": L.MX_TUNE_LU_TENSOR,
    "lu_grid": L.MX_TUNE_LU_GRID,
    "dots": L.MX_TUNE_DOTS,
    "coarse_inverse": L.MX_TUNE_COARSE_INVERSE,
    "local_tensor": L.MX_TUNE_LOCAL_TENSOR,
    "local_rhs_group": L.MX_TUNE_LOCAL_RHS_GROUP,
    "coarse_blocks": L.MX_TUNE_COARSE_BLOCKS,
}

# library defaults, written out so that a cached choice never depends on "0 = default"
DEFAULTS = {"lu_tensor": 0, "lu_grid": 0, "dots": 0, "coarse_inverse": 1, "local_tensor": 1, "local_rhs_group": 16,
            "coarse_blocks": 0}

FORMAT = 3


def candidates(info, cfg, name, allow_reduced=False):
    """Values of knob `name` worth timing for a problem with mx_info `info`, given the
    other knobs in `cfg`. An empty list means the knob has no effect on this problem."""
    mixed = info["precision"] == L.MX_MIXED
    coarse = info["n_coarse"] > 0
    if name == "lu_tensor":
        # 1 (a single TF32 product) changes the factors' accuracy: only on request
        return ([0, 3, 4, 1] if allow_reduced else [0, 3, 4]) if mixed else []
    if name == "lu_grid":
        # CTAs of the persistent LU (0: one per subdomain); only with the persistent LU
        persistent = cfg.get("lu_tensor", 0) in (0, 2)
        return [0, 152, 114, 76] if (mixed and persistent and info["n_sub"] > 152) else []
    if name == "dots":
        # the staged second pass applies to 2, 4, 8, 16 or 32 right-hand sides; the cost
        # measures it at the tuning batch's count, which the cache key records
        return [0, 1] if mixed else []
    if name == "coarse_inverse":
        return [1, 2, 0] if (mixed and coarse) else []
    if name == "local_tensor":
        return [1, 0] if mixed else []
    if name == "local_rhs_group":
        # the CUDA-core local solve; the tensor-core one takes its own groups, but falls back
        # to the CUDA cores above its half-bandwidth limit, which mx_info does not report
        return [16, 8, 4, 2, 1]
    if name == "coarse_blocks":
        sweeps = coarse and (not mixed or cfg.get("coarse_inverse", 1) == 0)
        return [0, 19, 38, 76, 152] if sweeps else []
    raise KeyError(name)


def cache_key(info, nrhs, device, tag=""):
    return "|".join([
        "v%d" % FORMAT, str(device), "nrhs=%d" % nrhs, "prec=%d" % info["precision"], "ndof=%d" % info["n_dof"],
        "nsub=%d" % info["n_sub"], "maxloc=%d" % info["max_local"], "nc=%d" % info["n_coarse"],
        "cband=%d" % info["coarse_band"], "tag=%s" % tag,
    ])


class Cache:
    """JSON file of tuned choices; a missing or unreadable file reads as empty."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        try:
            with open(path) as f:
                data = json.load(f)
            if isinstance(data, dict) and data.get("format") == FORMAT and isinstance(data.get("entries"), dict):
                self.entries = data["entries"]
        except (OSError, ValueError):
            pass

    def get(self, key):
        e = self.entries.get(key)
        if not isinstance(e, dict) or not isinstance(e.get("knobs"), dict):
            return None
        knobs = e["knobs"]
        if set(knobs) - set(KNOBS) or not all(isinstance(v, int) for v in knobs.values()):
            return None
        return e

    def put(self, key, entry):
        self.entries[key] = entry

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune-", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump({"format": FORMAT, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def apply(P, knobs):
    """Set every knob of `knobs` ({name: value}) on problem P (takes effect as each knob's
    documentation in include/mxas.h says: most at the next mx_factor)."""
    for name, v in knobs.items():
        P.set_tuning(KNOBS[name], int(v))


def default_rhs(n_dof, nrhs, seed=0):
    """Seeded complex Gaussian right-hand sides [nrhs, n_dof], on the GPU when torch has one."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((nrhs, n_dof)) + 1j * rng.standard_normal((nrhs, n_dof))
    try:
        import torch
        if torch.cuda.is_available():
            return torch.from_numpy(b).cuda()
    except ImportError:
        pass
    return b


def make_measure(P, rhs, tol=1e-6, restart=0, max_it=200, repeats=2, solves_per_factor=1.0):
    """Cost of a knob setting on problem P: factor, one warm-up solve, then the best of
    `repeats` timed solves. Returns (cost_ms or inf when a right-hand side fails to
    converge, details)."""

    def measure(knobs):
        apply(P, knobs)
        P.factor()
        factor_ms = P.timings()["factor_ms"]
        x = None
        best, its = float("inf"), None
        for r in range(repeats + 1):
            x, st, rc = P.solve(rhs, tol, restart, max_it, x=x)
            if rc != L.MX_OK or not all(s["converged"] for s in st):
                return float("inf"), {"factor_ms": factor_ms, "converged": False}
            if r > 0:
                best = min(best, P.timings()["solve_ms"])
                its = max(s["iterations"] for s in st)
        return factor_ms + solves_per_factor * best, {"factor_ms": factor_ms, "solve_ms": best,
                                                      "iterations": its, "converged": True}

    return measure


def search(info, measure, allow_reduced=False, min_gain=0.02, sweeps=1):
    """Coordinate search over KNOBS from DEFAULTS. `measure(knobs) -> (cost, details)`.
    Returns (best knobs, best cost, default cost, list of trials)."""
    cfg = dict(DEFAULTS)
    trials = []
    seen = {}

    def run(c):
        key = tuple(sorted(c.items()))
        if key not in seen:
            cost, det = measure(dict(c))
            seen[key] = cost
            trials.append({"knobs": dict(c), "cost_ms": cost, **det})
        return seen[key]

    base = run(cfg)
    if not np.isfinite(base):
        raise RuntimeError("the default knob setting does not converge on this problem; nothing to tune against")
    best = base
    for _ in range(sweeps):
        changed = False
        for name in KNOBS:
            for v in candidates(info, cfg, name, allow_reduced):
                if v == cfg[name]:
                    continue
                c = dict(cfg, **{name: v})
                cost = run(c)
                if cost < best * (1.0 - min_gain):
                    cfg, best, changed = c, cost, True
        if not changed:
            break
    return cfg, best, base, trials


def tune(P, nrhs=16, tol=1e-6, restart=0, max_it=200, cache_path=None, device=None, rhs=None, measure=None,
         allow_reduced=False, min_gain=0.02, sweeps=1, repeats=2, solves_per_factor=1.0, seed=0, tag=""):
    """Pick the knobs for problem P (built, factored or not), apply them and leave P
    factored under them. With `cache_path`, a cached choice for the same device, shape and
    right-hand-side count is applied without measuring, and a new choice is stored.
    Returns the cache entry: {"knobs", "cost_ms", "default_ms", "trials", "cached"}."""
    info = P.info()
    if device is None:
        try:
            import torch
            device = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
        except ImportError:
            device = "none"
    key = cache_key(info, nrhs, device, tag)
    cache = Cache(cache_path) if cache_path else None
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            apply(P, hit["knobs"])
            P.factor()
            return dict(hit, cached=True)
    if measure is None:
        if rhs is None:
            rhs = default_rhs(info["n_dof"], nrhs, seed)
        measure = make_measure(P, rhs, tol, restart, max_it, repeats, solves_per_factor)
    knobs, cost, base, trials = search(info, measure, allow_reduced, min_gain, sweeps)
    apply(P, knobs)
    P.factor()
    entry = {"knobs": knobs, "cost_ms": cost, "default_ms": base, "trials": len(trials),
             "tol": tol, "solves_per_factor": solves_per_factor}
    if cache is not None:
        cache.put(key, entry)
        cache.save()
    return dict(entry, cached=False, trial_log=trials)
