"""The C ABI library builds, loads without a GPU and exports every entry point of include/perc.h."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "perc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(perc_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("perc_rank", "perc_nstar", "perc_mass", "perc_smax_window", "perc_binomial_weights", "perc_pmax",
                 "perc_workspace_bytes", "perc_check",
                 "perc_status_string", "perc_bracket", "perc_mlp_train"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2607_18991_b300 import build, perc
    build.build()
    lib = perc.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", perc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (perc_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None
    assert set(perc.exported_symbols()) <= exported


def test_status_strings_without_gpu():
    from paper_2607_18991_b300 import perc
    assert perc.status_string(0) == "ok"
    assert "workspace" in perc.status_string(-2)
    assert perc.status_string(-99) == "unknown status"


def test_host_side_argument_checks_without_gpu():
    # invalid arguments are rejected before any CUDA call, so this runs on a CPU-only machine
    from paper_2607_18991_b300 import perc
    lib = perc.lib()
    assert lib.perc_rank(0, None, 1, None, None, None, 0, None) == -1
    assert lib.perc_rank(74, 1, 1, 1, 1, 1, 1 << 30, None) == -1
    assert lib.perc_nstar(None, 1, 8, None, None, None, None, None, 0, None) == -1
    assert lib.perc_mass(None, 1, 8, None, None, None, 0, None) == -1
    assert lib.perc_smax_window(None, 1, 8, 1, None, 4, 1, 1, 1, None) == -1
    assert lib.perc_smax_window(1, 1, 8, 1, None, 0, 1, 1, 1, None) == -1  # empty window
    assert lib.perc_smax_window(1, 1 << 20, 8, 1, None, 1 << 21, 1, 1, 1, None) == -1  # output over 2^40
    assert lib.perc_binomial_weights(None, 1, None, 1, 1, 1, 1, 1, None) == -1
    assert lib.perc_binomial_weights(1, 1, None, 1, 0, 1, 1, 1, None) == -1
    assert lib.perc_pmax(1, 1, 0, 1, 1, 1, None, 1, 1, 1, None) == -1
    assert lib.perc_pmax(1, None, 1, 1, 1, 1, None, 1, 1, 1, None) == -1
    assert lib.perc_workspace_bytes(7, 8, 1) == 0
    assert lib.perc_workspace_bytes(1, 0, 1) == 0
    assert lib.perc_workspace_bytes(1, 8, 1) > 8 * 8 ** 5
    # perc_nstar_min_axes: null pointers, no rows, axes outside 1..5
    assert lib.perc_nstar_min_axes(None, 4, 5, 1, None) == -1
    assert lib.perc_nstar_min_axes(1, 4, 5, None, None) == -1
    assert lib.perc_nstar_min_axes(1, 0, 5, 1, None) == -1
    assert lib.perc_nstar_min_axes(1, 4, 0, 1, None) == -1
    assert lib.perc_nstar_min_axes(1, 4, 6, 1, None) == -1
    # perc_microbench: unknown probe, null buffer, too small, no iterations
    import ctypes
    u = ctypes.c_double()
    assert lib.perc_microbench(9, 1, 1 << 20, 1, ctypes.byref(u), None) == -1
    assert lib.perc_microbench(1, None, 1 << 20, 1, ctypes.byref(u), None) == -1
    assert lib.perc_microbench(1, 1, 100, 1, ctypes.byref(u), None) == -1
    assert lib.perc_microbench(1, 1, 1 << 20, 0, ctypes.byref(u), None) == -1


def test_zone_word_layout():
    # the zone word packs the zones in bits 0..6 and the spanning axis in bits 8..10, as the header
    # defines it (PERC_ZONE_WORD)
    from paper_2607_18991_b300 import perc
    hdr = open(os.path.join(ROOT, "include", "perc.h")).read()
    assert re.search(r"#define PERC_AXIS_SHIFT 8u", hdr) and re.search(r"#define PERC_ZONE_BITS 0x7Fu", hdr)
    assert perc.AXIS_SHIFT == 8 and perc.NUM_AXES == 5
    assert int(perc.zone_word(127, 4)) == 127 | (4 << 8)
    assert list(perc.zone_word([1, 2], [0, 3])) == [1, 2 | (3 << 8)]
