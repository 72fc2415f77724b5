"""The oracle's translocation runs behind the exponent comparison
(tests/golden/oracle_transloc_eps2e-3.txt, written by
tests/golden/make_oracle_transloc.py): every line names the realisation the
script defines, and one short realisation re-run through the same script
reproduces its line exactly (FP64, one thread)."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _script():
    spec = importlib.util.spec_from_file_location("make_oracle_transloc",
                                                  os.path.join(GOLDEN, "make_oracle_transloc.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _lines(mod):
    rows = []
    for line in open(mod.OUT):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            assert len(f) == 7, line
            rows.append(tuple(int(x) for x in f[:6]))
    return rows


def test_lines_name_the_scripts_realisations():
    mod = _script()
    rows = _lines(mod)
    assert rows, "no oracle runs recorded"
    seen = set()
    for n, s, seed, state, t, steps in rows:
        assert n in mod.LENGTHS and 0 <= s < mod.SEEDS
        assert seed == 3000 + 1000 * n + s
        assert (n, s) not in seen
        seen.add((n, s))
        assert state in (0, 1, 2, 3, 4)
        assert 0 < steps <= mod.CAP + 25
        if state == 1:  # translocated: stepped in blocks of 25 up to the end
            assert 0 < t <= steps < t + 25
        else:
            assert t == -1


def test_a_short_realisation_reproduces_its_line():
    mod = _script()
    rows = {(n, s): (state, t, steps) for n, s, _, state, t, steps in _lines(mod)}
    if (50, 1) not in rows:
        pytest.skip("realisation (50, 1) not recorded")
    import oracle

    threads = oracle.max_threads()
    try:
        n, s, seed, state, t, steps, _ = mod.run_one((50, 1))  # one thread, as the script
    finally:
        oracle.set_threads(threads)
    assert (n, s, seed) == (50, 1, 3000 + 1000 * 50 + 1)
    assert (state, t, steps) == rows[(50, 1)]
