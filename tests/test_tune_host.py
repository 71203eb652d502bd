"""Fusion-depth table of the autotuner (host only, no GPU): the depth that
plan_create(-1) takes for (n, dtype), recorded entries, the cache file and the
PAULIROT_TUNE_CACHE variable."""
import os
import subprocess
import sys

import pytest

from paper_2602_09020_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def clean_table():
    """Remove the entries a test records (the table is process-wide)."""
    touched = []
    yield touched
    for n, dtype in touched:
        capi.plan_set_tuned_depth(n, dtype, -1)


def test_defaults_without_an_entry():
    assert capi.plan_tuned_depth(24, "c64") == (4, False)
    assert capi.plan_tuned_depth(24, "c128") == (3, False)
    # capped at n
    assert capi.plan_tuned_depth(2, "c64") == (2, False)
    assert capi.plan_tuned_depth(1, "c128") == (1, False)


def test_recorded_entries_and_removal(clean_table):
    clean_table += [(17, "c64"), (17, "c128"), (3, "c64")]
    capi.plan_set_tuned_depth(17, "c64", 2)
    capi.plan_set_tuned_depth(17, "c128", 5)
    capi.plan_set_tuned_depth(3, "c64", 5)
    assert capi.plan_tuned_depth(17, "c64") == (2, True)
    assert capi.plan_tuned_depth(17, "c128") == (5, True)
    assert capi.plan_tuned_depth(3, "c64") == (3, True)
    assert capi.plan_tuned_depth(18, "c64") == (4, False)  # per n
    capi.plan_set_tuned_depth(17, "c64", -1)
    assert capi.plan_tuned_depth(17, "c64") == (4, False)


@pytest.mark.parametrize("args", [(0, "c64", 2), (35, "c64", 2), (34, "c128", 2), (10, "c64", 0),
                                  (10, "c64", 6), (10, "c64", -2)])
def test_invalid_entries_are_rejected(args):
    with pytest.raises(capi.PauliRotError) as e:
        capi.plan_set_tuned_depth(*args)
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError):
        capi.plan_tuned_depth(0, "c64")


def test_cache_file_round_trip(tmp_path, clean_table):
    clean_table += [(20, "c64"), (21, "c128")]
    capi.plan_set_tuned_depth(20, "c64", 3)
    capi.plan_set_tuned_depth(21, "c128", 1)
    path = str(tmp_path / "tune.txt")
    capi.plan_tune_cache_save(path)
    lines = [l.split() for l in open(path) if not l.startswith("#")]
    assert ["c64", "20", "3"] in lines and ["c128", "21", "1"] in lines
    capi.plan_set_tuned_depth(20, "c64", -1)
    capi.plan_set_tuned_depth(21, "c128", -1)
    assert capi.plan_tuned_depth(20, "c64") == (4, False)
    capi.plan_tune_cache_load(path)
    assert capi.plan_tuned_depth(20, "c64") == (3, True)
    assert capi.plan_tuned_depth(21, "c128") == (1, True)
    # a missing file is an empty table
    capi.plan_tune_cache_load(str(tmp_path / "absent.txt"))
    assert capi.plan_tuned_depth(20, "c64") == (3, True)


@pytest.mark.parametrize("text", ["c64 20\n", "c32 20 3\n", "c64 20 9\n", "c64 40 3\n", "c64 20 3 x\n",
                                  "c64 twenty 3\n"])
def test_malformed_cache_changes_nothing(tmp_path, clean_table, text):
    clean_table += [(12, "c64"), (20, "c64")]
    capi.plan_set_tuned_depth(12, "c64", 2)
    path = tmp_path / "bad.txt"
    path.write_text("# header\nc64 12 5\n" + text)
    with pytest.raises(capi.PauliRotError) as e:
        capi.plan_tune_cache_load(str(path))
    assert e.value.code == capi.SV_EINVAL
    assert capi.plan_tuned_depth(12, "c64") == (2, True)  # the good line before it was not taken either
    assert capi.plan_tuned_depth(20, "c64") == (4, False)


def test_environment_cache_is_read_before_the_first_lookup(tmp_path):
    path = tmp_path / "env.txt"
    path.write_text("# fusion depth\nc64 19 2\n\nc128 19 4\n")
    code = ("from paper_2602_09020_gb300 import capi\n"
            "print(capi.plan_tuned_depth(19, 'c64'), capi.plan_tuned_depth(19, 'c128'),"
            " capi.plan_tuned_depth(20, 'c64'))\n")
    env = dict(os.environ, PAULIROT_TUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "(2, True) (4, True) (4, False)"


def test_concurrent_saves_leave_a_whole_cache(tmp_path):
    """Processes that save the table to one file at the same time each write
    their own temporary file and rename it over the cache, so the file is
    always one process's complete table."""
    path = tmp_path / "shared.txt"
    code = ("import sys\n"
            "from paper_2602_09020_gb300 import capi\n"
            "k = int(sys.argv[1])\n"
            "for n in range(10, 30):\n"
            "    capi.plan_set_tuned_depth(n, 'c64', 1 + (n + k) % 5)\n"
            "for _ in range(50):\n"
            "    capi.plan_tune_cache_save(sys.argv[2])\n")
    procs = [subprocess.Popen([sys.executable, "-c", code, str(k), str(path)], cwd=ROOT) for k in range(4)]
    assert all(p.wait(timeout=120) == 0 for p in procs)
    lines = [l.split() for l in path.read_text().splitlines() if not l.startswith("#")]
    assert len(lines) == 20
    assert sorted(int(n) for _, n, _ in lines) == list(range(10, 30))
    # one writer's table: every entry follows the same k
    offs = {(int(d) - 1 - int(n)) % 5 for _, n, d in lines}
    assert len(offs) == 1
    assert not list(tmp_path.glob("shared.txt.tmp*"))
