"""Autotuner of the y/z pass's launch shape (per padded size), with a JSON cache.

The y/z pass (the demagnetising product's y transforms and z sum, eq. 14) runs
either as one fused kernel per kx column or as the split pass (three kernels
through a buffer), whose z product works on ky blocks of a chosen size.  Which
is faster depends on the grid: the number of kx columns against the 148 SMs,
the planes per column, the block's shared memory.  ``autotune`` times every
candidate on the solver's own film with CUDA events (``mm_step_timed``, the y/z
class of kernels), keeps the fastest, and records it under the padded size in a
JSON file; ``mm_opts.tune_cache`` (``Solver(..., tune_cache=path)``) makes
``mm_create`` apply it, and ``apply_cached`` applies it to an existing solver.
The state, the clock and the step count of the solver are restored afterwards.
Results are identical for every candidate; only the time differs.
"""
import json
import os

__all__ = ["autotune", "apply_cached", "cache_key"]


def cache_key(solver) -> str:
    px, py, _ = solver.padded_dims()
    return f"{px}x{py}x{solver.grid[2]}:{solver.precision}"


def _candidates(solver):
    """(route, block) pairs: the fused kernel when a column fits one CTA, and the
    split pass with ky blocks 8, 16, 32, ... up to the largest that fits."""
    out = []
    try:
        solver.set_tuning(1, 0)
        out.append((1, 0))
    except Exception:
        pass
    if solver.precision == "fp32":
        solver.set_tuning(2, 0)
        kmax = solver.tuning()[1]
        solver.set_tuning(2, 4096)
        kmax = max(kmax, solver.tuning()[1])
        kb = 8
        while kb <= kmax:
            out.append((2, kb))
            kb *= 2
    solver.set_tuning(0, 0)
    return out


def autotune(solver, dt: float, cache: str = None, steps: int = 3) -> dict:
    """Time every candidate launch shape for ``steps`` steps of ``dt``; apply the
    fastest and (if ``cache`` is given) store it there.  Returns the record."""
    torch = solver.torch
    m = solver.get_m().clone()
    t0 = solver.time()
    timings = {}
    for route, kb in _candidates(solver):
        solver.set_tuning(route, kb)
        solver.set_m(m)
        solver.step_timed(1, dt)   # warm-up (first launches, L2)
        torch.cuda.synchronize()
        ms = solver.step_timed(steps, dt)[1] / steps
        timings[f"{route}:{kb}"] = ms
    best = min(timings, key=timings.get)
    route, kb = (int(v) for v in best.split(":"))
    solver.set_tuning(route, kb)
    solver.set_m(m)
    solver.set_time(t0)
    rec = {"yz_route": route, "zt_block": kb, "yz_ms_per_step": timings[best], "candidates": timings}
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[cache_key(solver)] = rec
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return rec


def apply_cached(solver, cache: str) -> bool:
    """Apply the launch shape stored for this solver's padded size; False if none."""
    if not os.path.exists(cache):
        return False
    with open(cache) as f:
        rec = json.load(f).get(cache_key(solver))
    if not rec:
        return False
    solver.set_tuning(rec["yz_route"], rec["zt_block"])
    return True
