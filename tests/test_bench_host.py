"""Host-side checks of bench.py and the autotuner, without a GPU.

- The reference arm (the oracle, timed on the host) prints one JSON line with
  the contract's keys: impl = reference, the arm's metric and unit, a
  cpu_baseline describing the run (whole solves on every host core) and an
  e2e object with zero copy bytes. The workload is shrunk to 129^2 here so
  that the check takes a second.
- The autotuner searches one knob at a time (each knob tuned with the others
  at their best so far), keeps the fastest candidate, and serves a repeated
  request for the same problem from its cache without timing again.
"""
import io
import json
import sys
import types
from contextlib import redirect_stdout

import pytest

import bench


def test_reference_arm_prints_the_contract_line(monkeypatch):
    monkeypatch.setattr(bench, "WORKLOAD", dict(bench.WORKLOAD, n=129))
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = types.SimpleNamespace(steps=2, warmup=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["metric"] == bench.METRIC and rec["higher_is_better"] is True
    assert rec["value"] > 0 and abs(rec["value"] * rec["ms_per_step"] - 1e3) < 1e-6 * 1e3
    import oracle
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] == oracle.host_cores()
    assert "whole FP64 oracle solve" in rec["cpu_baseline"]["sample"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    assert (rec["steps"], rec["warmup"]) == (2, 1)


def test_autotuner_coordinate_search_and_cache(monkeypatch, tmp_path):
    from paper_1406_5369_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "test-gpu")
    made = []

    class FakeSolver:
        def __init__(self, dim, n, **kw):
            self.kw = kw
            made.append(kw)

        def close(self):
            pass

    # time = (a - 2)^2 + (b - 3)^2 + 1: the search should land on a = 2, b = 3
    def fake_time(solver, f, tol, reps=3, stat="median"):
        assert stat == "min" and reps >= 3  # one disturbed timing must not decide
        kw = solver.kw
        return (kw["a"] - 2) ** 2 + (kw["b"] - 3) ** 2 + 1.0, 4

    monkeypatch.setattr(autotune, "time_solve", fake_time)
    import paper_1406_5369_gb300.solver as solver_mod
    monkeypatch.setattr(solver_mod, "Solver", FakeSolver)
    knobs = {"a": [0, 1, 2, 3], "b": [0, 3, 5]}
    best, table = autotune.tune(2, 65, None, 1e-8, knobs, base={"precision": "fp32_dc"})
    assert best == {"a": 2, "b": 3}
    assert len(made) == 4 + 3
    # b was searched with a at its best value
    assert all(m["a"] == 2 for m in made[4:])
    assert all(m["precision"] == "fp32_dc" for m in made)
    again, _ = autotune.tune(2, 65, None, 1e-8, knobs, base={"precision": "fp32_dc"})
    assert again == best and len(made) == 7  # served from the cache


def test_paper_gpu_times_in_bench_are_derived_from_table2():
    # bench.py quotes the paper's GPU times (context beside its own) as the
    # first column of Table 2 divided by the GPU speedup columns
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table2_runtimes.json")) as fh:
        rows = json.load(fh)["rows"]
    pairs = {("2D", "jacobi"): "laplacian_2d_jacobi", ("2D", "rbgs"): "laplacian_2d_gauss_seidel",
             ("3D", "jacobi"): "laplacian_3d_jacobi", ("3D", "rbgs"): "laplacian_3d_gauss_seidel"}
    for key, row in pairs.items():
        r = rows[row]
        d, f = bench.PAPER_TABLE2_GTX680_MS[key]
        assert abs(d - r[0] / r[4]) <= 0.05 and abs(f - r[0] / r[5]) <= 0.05, key
    for sm, row in (("jacobi", "complex_diffusion_2d_jacobi"), ("rbgs", "complex_diffusion_2d_gauss_seidel")):
        r = rows[row]
        d, f = bench.PAPER_TABLE2_CD_GTX680_MS[sm]
        assert abs(d - r[0] / r[4]) <= 1e-9 and abs(f - r[0] / r[5]) <= 1e-9, sm


def test_lfa_summary_of_the_3d_jacobi_cycle():
    out = bench.lfa_summary(3, "jacobi", 6.0 / 7.0, 2, 2)
    assert 0.2 < out["rho_two_grid_configured"] < 0.3
    assert out["rho_two_grid_lfa"] <= out["rho_two_grid_configured"] + 1e-12
    assert 0.5 <= out["omega_lfa"] <= 1.0


def test_final_error_against_the_converged_oracle():
    # a solution perturbed by a known vector: the reported relative error is
    # that vector's size, and the guaranteed bound from the residual covers it
    import numpy as np
    import oracle
    import synth
    n = 129
    f = synth.uniform_rhs(2, n, 5)
    H = oracle.Hierarchy(2, n, mt=True)
    H.set_rhs(f)
    H.solve(1e-13, 30)
    us = H.get_u()
    d = np.zeros_like(us)
    d[1:-1, 1:-1] = 1e-9 * np.max(np.abs(us)) * np.sin(np.arange(n - 2))[None, :]
    out = bench.final_error_vs_oracle({"x": us + d, "same": us.copy()}, H, f)
    assert out["same"]["rel_l2"] <= 1e-15 and out["same"]["rel_max"] <= 1e-15
    want = np.sqrt(np.sum(d * d)) / np.sqrt(np.sum(us * us))
    assert abs(out["x"]["rel_l2"] - want) <= 1e-3 * want
    assert out["x"]["rel_l2"] <= out["x"]["rel_l2_bound"]
    assert out["oracle"]["relres"] <= 1e-12
