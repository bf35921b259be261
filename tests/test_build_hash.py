"""The kernel source hash that ties recorded profiler counters to a kernel version: a
change of comments or blank space leaves it unchanged, a change of code does not."""
from paper_2411_14631_gb300 import build


def test_code_only_drops_comments_and_blank_space():
    a = "int x = 1; // one\n/* a\n block */ float y = 2.0f;\n\n"
    b = "int x = 1;   // another comment\nfloat y = 2.0f; /* trailing */"
    assert build._code_only(a) == build._code_only(b) == "int x = 1; float y = 2.0f;"


def test_code_change_changes_the_text():
    assert build._code_only("a = b + c; // x") != build._code_only("a = b - c; // x")


def test_source_hash_is_stable():
    h = build.source_hash()
    assert len(h) == 16 and h == build.source_hash()
