"""Host-side checks of the tile table that the autotuner fills (no GPU needed): export and
import round-trip, malformed text is rejected with the table unchanged, and a recorded
choice reaches the planner (the workspace size of an affected shape changes, and goes back
when the table is cleared)."""
import ctypes

import pytest

from tests.test_abi import make_desc


@pytest.fixture()
def lib():
    from paper_2011_06532_gb300 import _native

    _native.build()
    lib = _native.load()
    lib.tt_tune_clear()
    yield lib
    lib.tt_tune_clear()


def export(lib) -> str:
    n = ctypes.c_size_t(0)
    assert lib.tt_tune_export(None, 0, ctypes.byref(n)) == 0
    buf = ctypes.create_string_buffer(n.value)
    assert lib.tt_tune_export(buf, n.value, ctypes.byref(n)) == 0
    short = ctypes.create_string_buffer(1)
    assert lib.tt_tune_export(short, 1, ctypes.byref(n)) == 2
    return buf.value.decode()


def entries(text: str):
    return [ln for ln in text.splitlines() if ln.strip() and not ln.startswith("#")]


def test_round_trip_and_generation(lib):
    g0 = lib.tt_tune_generation()
    text = "# comment\n\n1 0 32 8 4 8 4 2 1\n2 1 4096 48 48 48 48 38 0\n"
    assert lib.tt_tune_import(text.encode()) == 0
    assert lib.tt_tune_generation() > g0
    got = entries(export(lib))
    assert sorted(got) == sorted(["1 0 32 8 4 8 4 2 1", "2 1 4096 48 48 48 48 38 0"])
    # importing the export gives the same table
    lib.tt_tune_clear()
    assert entries(export(lib)) == []
    assert lib.tt_tune_import("\n".join(got).encode()) == 0
    assert sorted(entries(export(lib))) == sorted(got)


@pytest.mark.parametrize("line", [
    "1 0 32 8 4 8 4 2",            # too few fields
    "1 0 32 8 4 8 4 2 1 9",        # too many
    "0 0 32 8 4 8 4 2 1",          # precision out of range
    "1 2 32 8 4 8 4 2 1",          # context out of range
    "1 0 0 8 4 8 4 2 1",           # I < 1
    "1 0 32 8 4 9 4 2 1",          # K0 > R0
    "1 0 32 8 4 8 5 2 1",          # K1 > R1
    "1 0 32 200 4 8 4 2 1",        # rank above the maximum
    "1 0 32 8 4 8 4 2000 1",       # P > 1024
    "1 0 32 8 4 8 4 -1 1",         # negative P
    "1 0 32 8 4 8 4 2 x",          # not a number
])
def test_malformed_text_rejected_table_unchanged(lib, line):
    assert lib.tt_tune_import(b"1 0 16 4 1 4 1 4 2\n") == 0
    before = export(lib)
    assert lib.tt_tune_import(("1 0 64 1 8 1 8 3 3\n" + line + "\n").encode()) == 1
    assert export(lib) == before


def test_recorded_choice_reaches_the_planner(lib):
    x = make_desc([64, 32, 16], [1, 8, 4, 1])
    n0, n1, n2 = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n0)) == 0
    # core 1 of x: I=32, R=(8,4), ranks after the orthogonalization sweep (8,4); 2 leaves
    assert lib.tt_tune_import(b"1 0 32 8 4 8 4 2 1\n") == 0
    assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n1)) == 0
    assert n1.value != n0.value
    # an entry for another precision or the batch context does not apply
    lib.tt_tune_clear()
    assert lib.tt_tune_import(b"2 0 32 8 4 8 4 2 1\n1 1 32 8 4 8 4 2 1\n") == 0
    assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n2)) == 0
    assert n2.value == n0.value
    lib.tt_tune_clear()
    assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n2)) == 0
    assert n2.value == n0.value


def test_autotune_workspace_covers_the_default_plan(lib):
    x = make_desc([64, 32, 16], [1, 8, 4, 1])
    n, m = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.tt_round_workspace_size(ctypes.byref(x), 1, ctypes.byref(n)) == 0
    assert lib.tt_autotune_workspace_size(ctypes.byref(x), 1, ctypes.byref(m)) == 0
    assert m.value >= n.value
    xs = (type(x) * 2)(x, make_desc([48, 48], [1, 6, 1]))
    assert lib.tt_round_batched_workspace_size(2, xs, 1, ctypes.byref(n)) == 0
    assert lib.tt_autotune_batched_workspace_size(2, xs, 1, ctypes.byref(m)) == 0
    assert m.value >= n.value
    bad = make_desc([4, 5], [2, 3, 1])
    assert lib.tt_autotune_workspace_size(ctypes.byref(bad), 1, ctypes.byref(m)) == 1
