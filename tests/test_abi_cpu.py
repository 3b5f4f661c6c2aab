"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/polyclean.h declares (no compute call is made here)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pc_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2406_01342_gb300 import abi, build
    path = build.build()
    assert os.path.exists(path)
    lib = abi.load()
    declared = _declared()
    assert declared == set(abi.EXPORTS), declared ^ set(abi.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.pc_abi_version() == abi.PC_ABI_VERSION


def test_header_cites_the_paper_for_each_entry_point():
    src = open(os.path.join(ROOT, "include", "polyclean.h")).read()
    for needle in ("Sect. 2.2", "Sect. 4.2", "Sect. 5.3", "Algorithm 2"):
        assert needle in src
