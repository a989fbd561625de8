"""The C ABI from plain C: tests/c/dry_run_consumer.c compiles as C11 against
include/ifgf.h alone, links the in-tree libifgf.so and sizes a plan on the host
(no GPU); its statistics equal those of the Python binding for the same points."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _points(n):
    """The consumer's point set, rebuilt here: equiangular cube-sphere with midpoint weights."""
    pts, w = [], []
    for f in range(6):
        for a in range(n):
            for b in range(n):
                u, v = -1 + (2 * a + 1) / n, -1 + (2 * b + 1) / n
                X, Y, s = np.tan(np.pi * u / 4), np.tan(np.pi * v / 4), (-1.0 if f % 2 else 1.0)
                p = np.zeros(3)
                ax = f // 2
                p[ax], p[(ax + 1) % 3], p[(ax + 2) % 3] = s, X, s * Y
                r = np.sqrt(1 + X * X + Y * Y)
                pts.append(p / r)
                w.append((np.pi / 4) ** 2 * (1 + X * X) * (1 + Y * Y) / r ** 3 * 4 / n ** 2)
    return np.array(pts), np.array(w)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_consumer_dry_run(tmp_path):
    from paper_2112_06316_gb300 import binding
    from paper_2112_06316_gb300 import build as _b

    lib = _b.build()
    exe = tmp_path / "consumer"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "dry_run_consumer.c"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-lifgf", "-Wl,-rpath," + os.path.dirname(lib), "-lm"],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe), "24", str(2 * np.pi)], check=True, capture_output=True, text=True).stdout
    lines = out.strip().splitlines()
    stats = dict(kv.split("=", 1) for kv in lines[0].split())
    x, w = _points(24)
    info = binding.dry_run(x, x, w, binding.Params(k=2 * np.pi))
    assert int(stats["N"]) == info["N"] == 6 * 24 * 24
    assert int(stats["D"]) == info["D"]
    assert int(stats["nrc"]) == sum(info["nrc"])
    assert int(stats["leaf_evals"]) == info["leaf_evals"] and int(stats["near_pairs"]) == info["near_pairs"]
    assert "5x8" in stats["orders"]
    assert lines[1].startswith("N=0 -> -1 (") and len(lines[1]) > len("N=0 -> -1 ()")
    assert lines[2].startswith("bad normal -> -1 (") and "unit" in lines[2]
