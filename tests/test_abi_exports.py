"""CPU check of the boundary: the compiled library loads and exports every
function that include/*.h declares (no compute call is made)."""
import ctypes
import glob
import os
import re

from paper_2309_02825_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lb[a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lb_create", "lb_set_theta0", "lb_step", "lb_macros", "lb_destroy", "lb_reduce",
                 "lb_sum_theta", "lb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
