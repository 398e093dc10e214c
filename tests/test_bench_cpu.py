"""Host-side checks of bench.py that need no GPU: the reference arm prints
one well-formed JSON line per configuration (the FP64 oracle on a bounded
sample, in the unit of the GPU arm), and the traffic records are keyed on
the sources of their own kernel."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*args):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", *args],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("args,unit,higher", [
    (["--config", "advdiff"], "unknowns/s", True),
    (["--config", "advdiff", "--cycle", "sawtooth"], "unknowns/s", True),
    (["--config", "timing3d", "--size", "128", "--cycle", "sawtooth"], "s", False),
    (["--config", "poisson2d"], "unknowns/s", True),
])
def test_reference_arm_line(args, unit, higher):
    d = _reference_line(*args)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == unit
    assert d["higher_is_better"] is higher
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["unit"] == unit
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and d["dtype"] == "f64"
    if "sawtooth" in args and "advdiff" in args:
        assert "L1" in d["metric"]


def test_traffic_records_follow_their_kernel_sources():
    sys.path.insert(0, ROOT)
    import bench
    for workload, tu in bench.TRAFFIC_TU.items():
        assert os.path.exists(os.path.join(ROOT, "paper_2402_17913_gb300", "csrc", tu))
        h = bench.source_hash(tu)
        assert len(h) == 12 and h != bench.source_hash()
        path = os.path.join(ROOT, "profiles", "traffic_%s.md" % workload)
        text = open(path).read()
        # the committed summary carries the hash of the sources it was taken on
        assert "src=" in text
    assert bench.recorded_traffic("no_such_workload", "up_fine") is None


def test_batched_batch_splits_over_ranks_by_work():
    """One batch split over the ranks: disjoint shares that together are the
    whole batch, balanced by sum of N^2; rank 0 of one rank is the whole
    single-GPU batch, with the same instances (masks and right-hand sides)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    whole = bench.Batched(count=12)
    assert whole.index == list(range(12)) and whole.job_units == whole.units
    parts = [bench.Batched(count=12, rank=r, world=3) for r in range(3)]
    idx = sorted(k for p in parts for k in p.index)
    assert idx == list(range(12))
    assert all(p.job_units == whole.job_units for p in parts)
    for p in parts:
        for k, rhs, solid in zip(p.index, p.rhs, p.solids):
            assert np.array_equal(rhs, whole.rhs[k]) and np.array_equal(solid, whole.solids[k])
    work = [sum(n * n for n, _ in p.shapes) for p in parts]
    assert max(work) - min(work) <= 512 * 512
    assert bench.shard_by_work([4, 3, 3, 2, 2, 2], 2) == [[0, 3, 4], [1, 2, 5]]


def test_paper_workload_parameters():
    """The timing workload and the implicit advection-diffusion test use the
    paper's printed parameters: a 10^3 cube centred at (32, 64, 64) in the
    128^3 domain with Re = 200 and dt = 0.1 (Sec. 3.4); (u, v) = (1, 1),
    nu = 2, dt = 50 (C = 50), a Gaussian of width 10 on 128^2 nodes
    (Sec. 3.2)."""
    sys.path.insert(0, ROOT)
    import bench
    t = bench.Timing3D(128)
    assert t.cells == (128, 128, 128) and t.block == 10 and t.centre == (32, 64, 64)
    assert abs(t.nu * 200.0 / (t.uin * t.block) - 1.0) < 1e-12 and t.dt == 0.1 and t.iters == 20
    assert t.paper_s[128] == (3.0, 165.0) and t.paper_s[256] == (11.0, 1275.0) and t.paper_s[512] == (34.0, 14376.0)
    a = bench.AdvDiff(128)
    assert a.shape == (128, 128) and (a.u, a.v, a.nu, a.dt, a.h) == (1.0, 1.0, 2.0, 50.0, 1.0)
    assert a.u * a.dt / a.h == 50.0 and a.gamma == 10.0


def test_gpus_flag_must_match_the_launch():
    """--gpus N under a launcher that started a different number of ranks is
    an error (the line would otherwise claim the wrong GPU count)."""
    env = dict(os.environ, WORLD_SIZE="1", RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--steps", "1"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode != 0 and "WORLD_SIZE" in out.stderr


def test_algorithmic_bytes_count_each_array_at_its_width():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algo_bytes_per_cell("up_fine", 2) == 13.0
    assert bench.algo_bytes_per_cell("up_fine", 3) == 12.5
    assert bench.algo_bytes_per_cell("up_fine", 3, "fp16") == 4 + 2 + 0.25 + 4
    assert bench.algo_bytes_per_cell("down_fine", 3, "bf16", masked=True) == 4 + 2 + 0.25 + 1
    assert bench.algo_bytes_per_cell("p_update", 3, "fp16") == 12
    assert bench.algo_bytes_per_cell("xr_update", 3) == 20
