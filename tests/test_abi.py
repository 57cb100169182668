"""The C-ABI library loads on a machine without a GPU and exports every
function that include/*.h declares; pure host calls behave as documented."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(tsat_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2511_07737_b300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 25
    for n in sorted(names):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2511_07737_b300", "libturbosat.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(tsat_[a-z0-9_]+)\b", out))
    assert names <= exported


def test_host_only_calls(lib):
    from paper_2511_07737_b300 import cnfgen
    from paper_2511_07737_b300 import turbosat as ts
    assert ts.strerror(-3).startswith("empty clause")
    hp = ts.hparams()
    assert abs(hp.lr0 - 0.1) < 1e-7 and hp.decay_period == 30 and hp.restart_period == 360
    assert ts.tsat_partial_k(1_000_000) == 100 and ts.tsat_partial_k(50) == 20 and ts.tsat_partial_k(7) == 7
    inst = cnfgen.planted_ksat(1000, 4200, 3, 0)
    b = ts.tsat_problem_bytes([(inst.n_vars, inst.clause_ptr, inst.lits)])
    assert b > 4200 * 3 * 4
    # malformed clause pointer is rejected on the host, before any device work
    import numpy as np
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_problem_bytes([(3, np.array([0, 2, 1]), np.array([1, 2]))])
    assert e.value.status == -1
