"""The sine and cosine polynomial constants of sq::box_muller
(include/squares_device.cuh) are the ones paper_2004_06278_gb300/csrc/fit_sincos.py
fits, and the fits are as accurate as the header states."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2004_06278_gb300", "csrc"))
import fit_sincos  # noqa: E402


def _header_poly(name):
    """Float literals of the fmaf chain that builds `name` (sp or cp), in the
    order they enter (highest power of t^2 first)."""
    src = open(os.path.join(ROOT, "include", "squares_device.cuh")).read()
    body = src[src.index("float2 box_muller(uint32_t hi, uint32_t lo)"):]
    lines = [ln for ln in body.splitlines() if re.search(rf"\b{name}\b = fmaf|float {name} = fmaf", ln)]
    lits = []
    for ln in lines:
        lits += [np.float32(float(x)) for x in re.findall(r"(-?\d\.\d+e[-+]\d+)f", ln)]
    return lits


def test_header_constants_match_the_fit():
    s, c = fit_sincos.fit()
    sp = _header_poly("sp")  # s3, s2, then s1, s0
    cp = _header_poly("cp")  # c3, c2, then c1 (c0 = 1 is the literal 1.0f)
    assert [float(x) for x in sp] == [float(s[3]), float(s[2]), float(s[1]), float(s[0])]
    assert [float(x) for x in cp] == [float(c[3]), float(c[2]), float(c[1])]
    assert float(c[0]) == 1.0


def test_fit_errors():
    es, ec = fit_sincos.max_errors()
    assert es < 3e-8 and ec < 6e-8, (es, ec)
