"""Planted mistakes in the oracle: each copy of ``oracle/squares_oracle.c``
below carries one plausible slip (a swapped addend, a dropped term, a wrong
rotation, a dropped round, ...). The pin battery of ``pins.py`` -- without
the arbitrary-precision route, which restates the definition -- must reject
every one of them. This shows the pins constrain the oracle and are not
satisfied by a wrong generator. CPU only; mutants are built with gcc in a
temporary directory."""
import ctypes
import os
import subprocess

import pytest

from tests import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "squares_oracle.c")

R1 = "x = middle_square_round(x, y);"
R2 = "x = middle_square_round(x, z);"

# (name, old text, new text, which occurrence of old text to replace)
# Occurrences count from 0 in file order: squares32's body precedes squares64's.
MUTANTS = [
    ("sq32 round 2 adds y", R2, "x = middle_square_round(x, y);", 0),
    ("sq32 round 1 adds z", R1, "x = middle_square_round(x, z);", 0),
    ("sq32 round 3 adds z", R1, "x = middle_square_round(x, z);", 1),
    ("sq32 round 3 dropped", R1, ";", 1),
    ("sq32 last round adds y", "const uint64_t last = x * x + z;",
     "const uint64_t last = x * x + y;", 0),
    ("sq32 returns low half", "return (uint32_t)(last >> 32);",
     "return (uint32_t)last;", 0),
    ("sq32 z = y + 1", "const uint64_t z = y + key;", "const uint64_t z = y + 1;", 0),
    ("sq32 y = ctr + key", "const uint64_t y = ctr * key;",
     "const uint64_t y = ctr + key;", 0),
    ("shift instead of rotate", "return (v << 32) | (v >> 32);", "return v >> 32;", 0),
    ("rotate by 31", "return (v << 32) | (v >> 32);", "return (v << 31) | (v >> 33);", 0),
    ("square without cross term", "return swap_halves(x * x + w);",
     "return swap_halves((x & 0xffffffffu) * (x & 0xffffffffu) + w);", 0),
    ("square keeps only the cross term",
     "return swap_halves(x * x + w);",
     "return swap_halves(((2 * (x & 0xffffffffu) * (x >> 32)) << 32) + w);", 0),
    ("sq64 round 1 adds z", R1, "x = middle_square_round(x, z);", 2),
    ("sq64 round 2 adds y", R2, "x = middle_square_round(x, y);", 1),
    ("sq64 round 3 dropped", R1, ";", 3),
    ("sq64 round 4 adds y", "const uint64_t t = x * x + z;",
     "const uint64_t t = x * x + y;", 0),
    ("sq64 round 5 adds z", "const uint64_t fifth = x * x + y;",
     "const uint64_t fifth = x * x + z;", 0),
    ("sq64 xor without shift", "return t ^ (fifth >> 32);", "return t ^ fifth;", 0),
    ("sq64 xors the rotated t", "return t ^ (fifth >> 32);", "return x ^ (fifth >> 32);", 0),
    ("sq64 fifth not squared", "const uint64_t fifth = x * x + y;",
     "const uint64_t fifth = x + y;", 0),
    ("sq64 z = y - key", "const uint64_t z = y + key;", "const uint64_t z = y - key;", 1),
]


def _mutate(src: str, old: str, new: str, occurrence: int) -> str:
    pos = -1
    for _ in range(occurrence + 1):
        pos = src.index(old, pos + 1)
    return src[:pos] + new + src[pos + len(old):]


def _build(tmp_path, name, text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_squares32.restype = ctypes.c_uint32
    lib.oracle_squares32.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_squares64.restype = ctypes.c_uint64
    lib.oracle_squares64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    m = (1 << 64) - 1
    return (lambda c, k: int(lib.oracle_squares32(c & m, k & m)),
            lambda c, k: int(lib.oracle_squares64(c & m, k & m)))


def test_unmutated_copy_passes(tmp_path):
    with open(SRC) as f:
        src = f.read()
    sq32, sq64 = _build(tmp_path, "clean", src)
    pins.run_scalar_battery(sq32, sq64)


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_rejected(tmp_path, name, old, new, occ):
    with open(SRC) as f:
        src = f.read()
    mutated = _mutate(src, old, new, occ)
    assert mutated != src
    sq32, sq64 = _build(tmp_path, "mutant", mutated)
    with pytest.raises(AssertionError):
        pins.run_scalar_battery(sq32, sq64)


# Planted mistakes in the Box-Muller pair; the battery of closed forms and
# polar identities must reject each.
BM_MUTANTS = [
    ("u1 = (hi + 1/2) / 2^32", "((double)hi + 1.0) / 4294967296.0", "((double)hi + 0.5) / 4294967296.0"),
    ("radius without the factor 2", "sqrt(-2.0 * log(u1))", "sqrt(-log(u1))"),
    ("cosine and sine exchanged", "*z0 = r * cos(theta);", "*z0 = r * sin(theta);"),
    ("angle pi lo / 2^32", "two_pi * ((double)lo", "0.5 * two_pi * ((double)lo"),
    ("sine negated", "*z1 = r * sin(theta);", "*z1 = -r * sin(theta);"),
    ("halves exchanged", "((double)hi + 1.0) / 4294967296.0", "((double)lo + 1.0) / 4294967296.0"),
]


def _build_bm(tmp_path, name, text):
    import numpy as np

    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_box_muller_f64.argtypes = [p, p, ctypes.c_uint64, p]

    def bm(hi, lo):
        hi = np.ascontiguousarray(hi, dtype=np.uint32)
        lo = np.ascontiguousarray(lo, dtype=np.uint32)
        out = np.empty((hi.size, 2), dtype=np.float64)
        lib.oracle_box_muller_f64(hi.ctypes.data, lo.ctypes.data, hi.size, out.ctypes.data)
        return out

    return bm


def test_unmutated_box_muller_passes(tmp_path):
    with open(SRC) as f:
        src = f.read()
    pins.run_box_muller_battery(_build_bm(tmp_path, "clean_bm", src))


@pytest.mark.parametrize("name,old,new", BM_MUTANTS, ids=[m[0] for m in BM_MUTANTS])
def test_box_muller_mutant_is_rejected(tmp_path, name, old, new):
    with open(SRC) as f:
        src = f.read()
    mutated = _mutate(src, old, new, 0)
    assert mutated != src
    with pytest.raises(AssertionError):
        pins.run_box_muller_battery(_build_bm(tmp_path, "mutant_bm", mutated))
