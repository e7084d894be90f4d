"""bench.py's host logic on the CPU: the reference arm's JSON line, the tape
event counts the walks' algorithmic work is computed from, and the reading of
the committed ncu summaries (a DRAM figure is reported only while the kernel
sources still hash to the one recorded with it)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-sample", "16"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "16 cells" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_walk_counts_from_a_tape():
    # INIT, REFACTOR, ITER, ITER, STEP(q1), RESCALE(q1), ITER, STEP(q2), REFACTOR, ITER, STEP(q2), REFACTOR
    kind = np.array([0, 4, 5, 5, 2, 1, 5, 2, 4, 5, 2, 4])
    q = np.array([1, 0, 0, 0, 1, 1, 0, 2, 0, 0, 2, 0])
    w = bench._walk_counts(kind, q)
    assert w["iter"] == 4 and w["inits"] == 1 and w["refactors"] == 3
    # the backward re-forms the matrices that govern accepted steps: the first
    # two steps share the REFACTOR at 1, the third has the one at 8; the
    # trailing REFACTOR governs no step
    assert w["ranges"] == 2
    assert w["step_q"].tolist() == [1.0, 2.0, 2.0] and w["rescale_q"].tolist() == [1.0]


def test_profiled_figure_follows_the_source_hash(tmp_path):
    sha = bench._kernel_sha()
    assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)
    p = tmp_path / "summary.md"
    p.write_text(f"# x\n\ndram_bytes_per_launch: 6406656\nsource_sha256: `{sha}`\n")
    assert bench._profiled(str(p)) == 6406656.0
    p.write_text("# x\n\ndram_bytes_per_launch: 6406656\nsource_sha256: `0000000000000000`\n")
    assert bench._profiled(str(p)) is None
    assert bench._profiled(str(tmp_path / "missing.md")) is None


@pytest.mark.parametrize("name", ["solve_kernel_fp64_persistent_tropo10k.md", "solve_kernel_fp32lu_persistent_tropo10k.md",
                                  "solve_kernel_fp64_plain_tropo10k.md", "adjoint_kernel_tropo2k.md",
                                  "tangent_kernel_tropo2k.md"])
def test_committed_summaries_carry_a_figure_and_a_hash(name):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    keys = {l.split(":", 1)[0].strip() for l in text.splitlines() if ":" in l}
    assert {"dram_bytes_per_launch", "source_sha256"} <= keys
    assert "--clock-control none" in text
