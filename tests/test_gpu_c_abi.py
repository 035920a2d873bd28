"""A plain C program grows two robots, continues them from their state,
prunes planner states and synthesises a design, through the C ABI alone."""
import subprocess

import pytest

from test_abi import _build_c_demo

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_c_caller_grows_robots(tmp_path):
    out = subprocess.run([_build_c_demo(tmp_path)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    rows = [line.split() for line in out.stdout.strip().splitlines()]
    extra = {r[0]: r[1:] for r in rows[2:]}
    rows = rows[:2]
    assert [r[0] for r in rows] == ["ok", "ok"] and [int(r[1]) for r in rows] == [12, 12]
    # relaxing an equilibrium with the length held moves the tip by at most the tolerance
    assert float(extra["relax"][0]) <= 1e-6 * 12 * 0.02 * 3
    assert extra["prune"] == ["0", "1", "1"]
    ip, il, th = int(extra["synth"][0]), int(extra["synth"][1]), float(extra["synth"][2])
    assert ip >= 0 and 0 <= il < 61 and abs(th - 0.03) <= 0.004
    x0, y0 = float(rows[0][2]), float(rows[0][3])
    assert abs(x0 - 12 * 0.02) < 1e-6 and abs(y0) < 1e-7  # unactuated, free space: straight
    assert float(rows[1][3]) > 1e-3  # the actuator on side +1 bends the robot toward +y
