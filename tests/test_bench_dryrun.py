"""bench.py's configuration sweep, incompressible part, dry-run on the CPU (tests/bench_dryrun.py):
the rows and the JSON line are well formed."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_incompressible_sweep_part_dry_run():
    r = subprocess.run([sys.executable, os.path.join(HERE, "bench_dryrun.py")], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    rows = line["sweep"]["inc"]
    assert len(rows) == 10 and line["steps"] == 10
    assert {row["method"] for row in rows} == {"ga-ngmres", "rpgd"}
    for row in rows:
        assert row["n"] == [256, 256] and row["nt"] == 16 and row["alpha"] == 1e-4
        assert row["det_min"] == row["det_max"] == 1.0
