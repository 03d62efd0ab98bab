"""The polynomial constants of sq::box_muller (include/squares_device.cuh)
are the ones paper_2004_06278_gb300/csrc/fit_box_muller.py fits, and the
fits are as accurate as the header states."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2004_06278_gb300", "csrc"))
import fit_box_muller as fit  # noqa: E402


def _header_chain(name):
    """Float literals of the fmaf chain that builds `name` (p, sp or cp) in
    sq::box_muller, in the order they enter (highest power first)."""
    src = open(os.path.join(ROOT, "include", "squares_device.cuh")).read()
    body = src[src.index("float2 box_muller(uint32_t hi, uint32_t lo)"):]
    body = body[:body.index("\n}\n")]
    lits = []
    for ln in body.splitlines():
        if re.search(rf"\b{name} = fmaf", ln):
            lits += [np.float32(float(x)) for x in re.findall(r"(-?\d\.\d+e[-+]\d+)f", ln)]
    return [float(x) for x in lits]


def test_sin_cos_constants_match_the_fit():
    s, c = fit.fit()
    assert _header_chain("sp") == [float(s[3]), float(s[2]), float(s[1]), float(s[0])]
    assert _header_chain("cp") == [float(c[3]), float(c[2]), float(c[1])]
    assert float(c[0]) == 1.0  # the chain's last addend is the literal 1.0f


def test_atanh_constants_match_the_fit():
    h = fit.fit_atanh()
    want = [float(np.float32(-4) * h[2]), float(np.float32(-4) * h[1]), float(np.float32(-4) * h[0])]
    assert _header_chain("p") == want


def test_fit_errors():
    es, ec, eh = fit.max_errors()
    assert es < 3e-8 and ec < 6e-8 and eh < 4e-8, (es, ec, eh)
