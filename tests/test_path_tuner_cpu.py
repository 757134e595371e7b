"""Host side of the path tuner (stab_path_*): defaults, the cache keyed by GPU
name and n, its text file, and rejection of malformed entries.  No GPU."""
import ctypes
import os

import pytest

from paper_2502_10685_gb300 import _lib


@pytest.fixture
def L():
    lib = _lib.load()
    lib.stab_path_clear()
    yield lib
    lib.stab_path_clear()


def choice(**kw):
    c = _lib.StabPathChoice()
    c.resident, c.resident_adjoint, c.gen_cut, c.tile_limit, c.tuned = 1, 1, 0.5, 1 << 17, 1
    c.gen_parts = 2
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def lookup(L, name, n):
    out = _lib.StabPathChoice()
    rc = L.stab_path_lookup(name.encode(), n, ctypes.byref(out))
    return rc, out


def test_defaults(L):
    for n in range(1, 13):
        c = _lib.StabPathChoice()
        assert L.stab_path_defaults(n, ctypes.byref(c)) == 0
        assert (c.resident, c.resident_adjoint, c.tile_limit, c.tuned) == (1, 1, 1 << 17, 0)
        assert c.gen_parts == 2
        assert c.gen_cut == (0.56 if n == 4 else 0.5)
    c = _lib.StabPathChoice()
    assert L.stab_path_defaults(0, ctypes.byref(c)) == -2
    assert L.stab_path_defaults(13, ctypes.byref(c)) == -2


def test_store_and_lookup_keyed_by_gpu_and_n(L):
    assert lookup(L, "GPU A", 5)[0] == -7                 # STAB_E_STATE: no entry
    assert L.stab_path_store(b"GPU A", 5, ctypes.byref(choice(resident=0))) == 0
    assert L.stab_path_store(b"GPU A", 6, ctypes.byref(choice(resident_adjoint=0))) == 0
    assert L.stab_path_store(b"GPU B", 5, ctypes.byref(choice(tile_limit=7))) == 0
    rc, c = lookup(L, "GPU A", 5)
    assert rc == 0 and c.resident == 0 and c.resident_adjoint == 1
    rc, c = lookup(L, "GPU A", 6)
    assert rc == 0 and c.resident == 1 and c.resident_adjoint == 0
    rc, c = lookup(L, "GPU B", 5)
    assert rc == 0 and c.tile_limit == 7 and c.resident == 1
    assert lookup(L, "GPU B", 6)[0] == -7
    # a later store replaces the entry
    assert L.stab_path_store(b"GPU A", 5, ctypes.byref(choice(gen_cut=0.62))) == 0
    rc, c = lookup(L, "GPU A", 5)
    assert rc == 0 and c.gen_cut == 0.62 and c.resident == 1
    assert L.stab_path_clear() == 0
    assert lookup(L, "GPU A", 5)[0] == -7


@pytest.mark.parametrize("bad", [dict(resident=2), dict(resident_adjoint=-1),
                                 dict(gen_cut=0.2), dict(gen_cut=0.71),
                                 dict(gen_cut=float("nan")), dict(tile_limit=-1),
                                 dict(tuned=3), dict(gen_parts=1), dict(gen_parts=4)])
def test_store_rejects_values_out_of_range(L, bad):
    assert L.stab_path_store(b"GPU A", 4, ctypes.byref(choice(**bad))) == -1
    assert lookup(L, "GPU A", 4)[0] == -7


def test_store_rejects_bad_names_and_n(L):
    for name in (b"", b"a\tb", b"a\nb", b"x" * 256):
        assert L.stab_path_store(name, 4, ctypes.byref(choice())) == -1
    assert L.stab_path_store(b"GPU A", 0, ctypes.byref(choice())) == -2
    assert L.stab_path_store(b"GPU A", 13, ctypes.byref(choice())) == -2


def test_file_round_trip(L, tmp_path):
    L.stab_path_store(b"NVIDIA GB300", 4, ctypes.byref(choice(gen_cut=0.46, gen_parts=3)))
    L.stab_path_store(b"NVIDIA GB300", 6, ctypes.byref(choice(resident=0, tile_limit=0)))
    L.stab_path_store(b"Other GPU", 8, ctypes.byref(choice(tile_limit=1 << 20, tuned=0)))
    f = str(tmp_path / "paths.tsv")
    assert L.stab_path_save(f.encode()) == 0
    lines = open(f).read().splitlines()
    assert len(lines) == 3 and all(len(ln.split("\t")) == 8 for ln in lines)
    L.stab_path_clear()
    assert lookup(L, "NVIDIA GB300", 4)[0] == -7
    assert L.stab_path_load(f.encode()) == 0
    rc, c = lookup(L, "NVIDIA GB300", 4)
    assert rc == 0 and c.gen_cut == 0.46 and c.gen_parts == 3 and c.tuned == 1
    rc, c = lookup(L, "NVIDIA GB300", 6)
    assert rc == 0 and c.resident == 0 and c.tile_limit == 0 and c.gen_parts == 2
    rc, c = lookup(L, "Other GPU", 8)
    assert rc == 0 and c.tile_limit == 1 << 20 and c.tuned == 0


def test_malformed_file_rejected_whole(L, tmp_path):
    L.stab_path_store(b"Kept", 5, ctypes.byref(choice(resident=0)))
    good = "NVIDIA GB300\t4\t1\t1\t0.56\t131072\t1\t2\n"
    for bad in ("NVIDIA GB300\t4\t1\t1\t0.56\n",                     # fields missing
                "NVIDIA GB300\t4\t1\t1\t0.56\t131072\t1\n",           # the parts missing
                "NVIDIA GB300\t4\t1\t1\t0.56\t131072\t1\t2\textra\n",  # a field too many
                "NVIDIA GB300\t13\t1\t1\t0.56\t131072\t1\t2\n",         # n out of range
                "NVIDIA GB300\t4\t1\t1\t0.9\t131072\t1\t2\n",           # cut out of range
                "NVIDIA GB300\t4\t1\t1\t0.56\t131072\t1\t5\n",          # parts out of range
                "no tab at all\n"):
        f = tmp_path / "bad.tsv"
        f.write_text(good + bad)
        assert L.stab_path_load(str(f).encode()) == -1, bad
        assert lookup(L, "NVIDIA GB300", 4)[0] == -7              # nothing taken
        rc, c = lookup(L, "Kept", 5)
        assert rc == 0 and c.resident == 0                      # the cache as it was
    assert L.stab_path_load(str(tmp_path / "missing.tsv").encode()) == -7


def test_cache_file_named_by_the_environment_is_read_at_first_lookup(tmp_path):
    """STAB_PATH_CACHE: a fresh process reads the named file before its first
    lookup (so a tuned choice carries over between processes); a malformed
    file is ignored and the cache starts empty."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    good = tmp_path / "paths.tsv"
    good.write_text("NVIDIA GB300\t6\t0\t0\t0.5\t131072\t1\t2\n"
                    "NVIDIA GB300\t4\t1\t1\t0.59\t131072\t1\t2\n")
    bad = tmp_path / "bad.tsv"
    bad.write_text("NVIDIA GB300\t6\t0\t0\t0.5\n")
    code = ("import ctypes, sys; sys.path.insert(0, %r)\n"
            "from paper_2502_10685_gb300 import _lib\n"
            "L = _lib.load(build_if_missing=False)\n"
            "c = _lib.StabPathChoice()\n"
            "rc6 = L.stab_path_lookup(b'NVIDIA GB300', 6, ctypes.byref(c)); r6 = c.resident\n"
            "rc4 = L.stab_path_lookup(b'NVIDIA GB300', 4, ctypes.byref(c)); cut = c.gen_cut\n"
            "print(rc6, r6, rc4, cut)\n" % root)
    env = dict(os.environ, STAB_PATH_CACHE=str(good))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["0", "0", "0", "0.59"]
    env = dict(os.environ, STAB_PATH_CACHE=str(bad))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split()[0] == "-7" and out.stdout.split()[2] == "-7"
