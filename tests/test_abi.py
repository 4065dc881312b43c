"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lfc.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lfc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lfc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2310_09467_gb300 import build, lfc
    so = build.build()
    lib = ctypes.CDLL(so)
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(lfc.EXPORTS) == declared


def test_pure_host_entry_points():
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    lib = lfc.load()
    assert lib.lfc_status_string(0) == b"ok"
    # container bound covers header + one worst-case stream per block
    one = lfc.max_stream_bytes(720000)
    assert one > 720000
    n = 2 * 2040 * 2040
    nb = -(-n // 720000)
    assert lfc.max_compressed_bytes(2040, 2040) >= 40 + 4 * nb + nb * 0 + (nb - 1) * one
    # invalid plan configurations are rejected before any device work
    cfg = lfc.Config()
    cfg.width, cfg.height, cfg.pitch, cfg.max_frames = 100, 100, 13, 1
    h = ctypes.c_void_p()
    assert lib.lfc_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1  # 100 % 13 != 0
    cfg.width, cfg.height, cfg.pitch = 104, 104, 13
    cfg.block_bytes = 720001
    assert lib.lfc_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1


def test_oracle_and_library_share_nothing():
    """The oracle and the CUDA path share no code: neither imports or
    includes the other."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "paper_2310_09467_gb300", "**", "*"), recursive=True):
        if os.path.isfile(f) and f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
            txt = open(f).read()
            assert "oracle" not in re.sub(r"#.*|//.*", "", txt).replace("the oracle", ""), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")) + glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        txt = open(f).read()
        assert "paper_2310_09467_gb300" not in txt and "lfc.h" not in txt, f
