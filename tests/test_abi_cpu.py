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


def test_plan_create_rejects_bad_arguments_without_a_gpu():
    """pc_plan_create checks every argument before its first CUDA call: each
    bad value returns PC_ERR_INVALID_ARG with a message naming it (M = 0, so
    no device pointer is needed; no GPU is touched)."""
    import ctypes
    import math

    from paper_2406_01342_gb300 import abi
    lib = abi.load()

    def create(N=64, fov=math.radians(2.0), version=abi.PC_ABI_VERSION, **opt):
        o = abi.pc_plan_opts(version, opt.get("kernel_width", 0), opt.get("tile", 0),
                             opt.get("max_planes", 0), opt.get("grid_mode", 0), opt.get("autotune", 0),
                             opt.get("fft_kernel", 0))
        h = ctypes.c_void_p()
        rc = lib.pc_plan_create(None, ctypes.c_int64(0), N, ctypes.c_double(fov), ctypes.byref(o), None,
                                ctypes.byref(h))
        return rc, lib.pc_last_error().decode()

    cases = [(dict(version=abi.PC_ABI_VERSION - 1), "version"), (dict(N=63), "N ="), (dict(N=8), "N ="),
             (dict(fov=0.0), "fov_rad"), (dict(fov=2.0), "fov_rad"), (dict(kernel_width=3), "kernel_width"),
             (dict(kernel_width=9), "kernel_width"), (dict(tile=16), "tile"), (dict(max_planes=5000), "max_planes"),
             (dict(grid_mode=4), "grid_mode"), (dict(autotune=2), "autotune"), (dict(fft_kernel=2), "fft_kernel")]
    for kw, needle in cases:
        rc, msg = create(**kw)
        assert rc == abi.PC_ERR_INVALID_ARG, (kw, rc, msg)
        assert needle in msg, (kw, msg)


def test_profile_classes_are_known_by_name_without_a_gpu():
    """pc_profile_begin_classes accepts every kernel class the library times
    (the degridding's FFT passes and its interpolation separately) and
    rejects an unknown name; with nothing launched, pc_profile_end reports no
    class (host bookkeeping only, no GPU is touched)."""
    from paper_2406_01342_gb300 import abi, build
    build.build()
    abi.load()
    classes = ["grid", "fft_rows", "fft_cols", "residual", "gram_fp32", "gram_finalize", "apgd", "select", "misc",
               "gram_tc", "gram_thin", "dict_corr", "dict_columns", "phase_gen", "apgd_op", "degrid", "degrid_fft"]
    abi.pc_profile_begin(",".join(classes))
    assert abi.pc_profile_end() == {}
    try:
        abi.pc_profile_begin("degrid_interp")
    except abi.PcError as e:
        assert e.status == abi.PC_ERR_INVALID_ARG
    else:
        raise AssertionError("an unknown class name was accepted")
    assert abi.pc_profile_end() == {}


def test_resume_arguments_are_checked_by_the_binding_without_a_gpu():
    """The binding passes a resume state only as device tensors with one
    weight per index (pc_solve reads them on the device); host tensors and a
    length mismatch are refused before any library call, and the options
    struct carries the state's size and iteration index."""
    import pytest
    import torch
    from paper_2406_01342_gb300 import abi
    idx = torch.tensor([3, 5], dtype=torch.int32)
    x = torch.tensor([1.0, 2.0], dtype=torch.float32)
    with pytest.raises(ValueError):
        abi._solve_opts(init_idx=idx, init_x=x, init_k=2)          # host tensors
    with pytest.raises(ValueError):
        abi._solve_opts(init_idx=idx, init_x=x[:1])                # one weight missing
    o = abi._solve_opts()
    assert o.init_S == 0 and o.init_k == 0 and not o.init_idx and not o.init_x
    assert o.version == abi.PC_ABI_VERSION
