"""The C-ABI library builds for sm_103a, loads, and exports every function
include/eap.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "eap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(eap_[a-z0-9_]+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("eap_nn1", "eap_nn1_host", "eap_pairwise", "eap_pairs", "eap_lb_keogh", "eap_serve_create",
                 "eap_serve_add_refset", "eap_serve_submit", "eap_serve_poll", "eap_serve_destroy", "eap_strerror"):
        assert must in names, must


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2102_05221_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in include/eap.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (eap_[a-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_library_targets_sm_103a_and_has_no_host_fallback():
    # The package has no CPU implementation of the path to fall back to: every
    # distance entry point is a symbol of libeap.so, compiled for sm_103a only.
    from paper_2102_05221_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    import paper_2102_05221_gb300.eap as E
    src = open(E.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_strerror_and_defaults_without_a_gpu():
    from paper_2102_05221_gb300 import eap
    lib = eap.load()
    assert lib.eap_strerror(-1) == b"invalid argument"
    p = eap.params("twe")
    assert abs(p.twe_nu - 0.001) < 1e-9 and p.twe_lambda == 1.0 and p.prune == 1
    p = eap.params("cdtw")
    assert abs(p.window_ratio - 0.1) < 1e-7 and p.window == -1


def test_params_layout_matches_the_header():
    # eap_params_default writes exactly sizeof(eap_params) bytes: the ctypes
    # mirror must have the same size, and the derivative flag defaults to 0.
    from paper_2102_05221_gb300 import eap
    lib = eap.load()
    n = ctypes.sizeof(eap.eap_params)
    buf = (ctypes.c_uint8 * (n + 16))(*([0xAB] * (n + 16)))
    lib.eap_params_default(ctypes.cast(buf, ctypes.POINTER(eap.eap_params)), 0)
    assert bytes(buf[n:]) == b"\xab" * 16
    p = eap.eap_params.from_buffer_copy(bytes(buf[:n]))
    assert p.derivative == 0 and p.prune == 1 and p.kind == 0
    assert eap.params("msm", derivative=1).derivative == 1
