"""The traffic digest follows the kernels' code: an edited comment or
indentation keeps a recorded DRAM-traffic figure, an edited line of code
voids it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _digest(tmp_path, text):
    p = tmp_path / "k.cu"
    p.write_text(text)
    return bench.sources_digest([str(p)])


def test_comments_and_blank_lines_do_not_change_the_digest(tmp_path):
    code = "int f(int x) {\n    return x + 1;\n}\n"
    commented = "// one\nint f(int x) {  // two\n\n    /* three\n       lines */ return x + 1;\n}\n"
    assert _digest(tmp_path, code) == _digest(tmp_path, commented)


def test_a_code_change_changes_the_digest(tmp_path):
    assert _digest(tmp_path, "int f(int x) { return x + 1; }\n") != _digest(tmp_path, "int f(int x) { return x + 2; }\n")

