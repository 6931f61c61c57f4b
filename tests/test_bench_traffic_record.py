"""The traffic record of bench.py: the stepper-code digest it is keyed on ignores line comments and
nothing else, and the recorded DRAM bytes of the default launch are plausible against the
algorithmic bytes (no GPU needed)."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture()
def source_copy(tmp_path, monkeypatch):
    """bench's stepper sources copied under tmp_path, with bench.ROOT pointing there."""
    for p in bench.STEPPER_SOURCES:
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _edit(path, fn):
    text = path.read_text(encoding="utf-8")
    path.write_text(fn(text), encoding="utf-8")


def test_digest_of_the_copy_equals_the_tree(source_copy):
    here = bench.stepper_digest()
    assert len(here) == 16
    assert here == bench.stepper_digest()  # deterministic


def test_comment_edits_keep_the_digest(source_copy):
    before = bench.stepper_digest()
    target = source_copy / bench.STEPPER_SOURCES[1]
    _edit(target, lambda t: "// a new leading comment line\n\n" + t.replace("\n", "   \n", 3))
    _edit(target, lambda t: t.replace("// ", "// reworded: ", 5))
    assert bench.stepper_digest() == before


def test_code_edits_change_the_digest(source_copy):
    before = bench.stepper_digest()
    target = source_copy / bench.STEPPER_SOURCES[1]
    text = target.read_text(encoding="utf-8")
    i = text.index("T(1.5)")
    target.write_text(text[:i] + "T(1.25)" + text[i + len("T(1.5)"):], encoding="utf-8")
    assert bench.stepper_digest() != before


def test_no_double_slash_inside_a_string_literal():
    """The digest cuts each line at its first '//': that must start a comment, never sit inside a
    string literal (an inline-PTX string, say), or a code edit there could go unnoticed."""
    for p in bench.STEPPER_SOURCES:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            for k, line in enumerate(f, 1):
                head = line.split("//", 1)[0]
                if "//" in line:
                    assert head.count('"') % 2 == 0, f"{p}:{k}: '//' inside a string literal"


def test_recorded_traffic_is_plausible():
    """The record is keyed on the default FP32 launch shape; its DRAM bytes per launch of the 64^3 x 64
    workload lie between 85% of the algorithmic bytes (written lines may still sit in L2 when the
    kernel ends) and 101% (no re-reads)."""
    wl = bench.WORKLOAD
    assert (wl["N"], wl["M"], wl["precision"], wl["pattern"]) == (64, 64, "fp32", "pull")
    algorithmic = 2 * 19 * 4 * wl["M"] * wl["N"] ** 3
    t = bench.NCU_TRAFFIC
    assert len(t["sha256"]) == 16 and t["launch"] == (3, 2, 128)
    assert 0.85 * algorithmic <= t["bytes_per_launch"] <= 1.01 * algorithmic
