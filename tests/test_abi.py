"""CPU-only checks of the C ABI library: it builds for sm_103a, loads without
a GPU, exports every function include/rsa.h declares, and validates
arguments on the host.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_06800_gb300 import build, rsa
    build.build()
    return rsa.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "rsa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsa_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rsa_create", "rsa_run_batch", "rsa_results", "rsa_destroy", "rsa_last_error",
              "rsa_workspace_bytes", "rsa_bind_workspace", "rsa_run_seeds", "rsa_run_keys"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1810_06800_gb300 import rsa
    for name in _declared():
        assert callable(getattr(rsa, name)), name


def test_create_validates_arguments(lib):
    from paper_1810_06800_gb300 import rsa
    for L, k in [(0, 0), (4, 0), (4, 5), (40000, 4)]:
        with pytest.raises(rsa.RSAError) as e:
            rsa.rsa_create(L, k, 1)
        assert e.value.code == rsa.RSA_EINVAL
    h = rsa.rsa_create(64, 4, 1)
    rsa.rsa_destroy(h)
    assert lib.rsa_create(64, 4, 1, None) == rsa.RSA_EINVAL


def test_workspace_bytes_is_monotone(lib):
    from paper_1810_06800_gb300 import rsa
    a = rsa.rsa_workspace_bytes(64, 4, 1)
    b = rsa.rsa_workspace_bytes(64, 4, 10)
    c = rsa.rsa_workspace_bytes(1024, 32, 1)
    assert 0 < a < b and c > a
    # about 13 bytes of lattice state per cell plus the contact graph
    assert c < 40 * 1024 * 1024


def test_results_before_run_is_a_state_error(lib):
    from paper_1810_06800_gb300 import rsa
    h = rsa.rsa_create(8, 2, 1)
    with pytest.raises(rsa.RSAError) as e:
        rsa.rsa_results(h, 1)
    assert e.value.code in (rsa.RSA_ESTATE, rsa.RSA_EINVAL)
    rsa.rsa_destroy(h)


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1810_06800_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "rsa_oracle" not in txt, f
    # and the oracle does not use the product path
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_1810_06800_gb300" not in txt, f
            assert "from paper_1810_06800_gb300" not in txt and "librsa_gb300" not in txt, f


def test_host_settings_validate_on_the_cpu(lib):
    # handle settings are host-side checks: 128-thread window CTAs need the
    # argmin-offset long-k path with 2048- or 4096-cell spans; 0 restores the
    # shape's default; rounds per check must be 1 .. 64
    from paper_1810_06800_gb300 import rsa
    for L, k, ok128 in [(32768, 4096, True), (8192, 512, True), (4096, 64, True),
                        (2048, 256, True), (1024, 32, False), (1024, 64, False),
                        (100, 3, False), (4096, 3500, False)]:
        h = rsa.rsa_create(L, k, 1)
        try:
            if ok128:
                rsa.rsa_set_window_threads(h, 128)
            else:
                with pytest.raises(rsa.RSAError) as e:
                    rsa.rsa_set_window_threads(h, 128)
                assert e.value.code == rsa.RSA_EINVAL
            rsa.rsa_set_window_threads(h, 256)
            rsa.rsa_set_window_threads(h, 0)
            for bad in (64, 512, 1):
                with pytest.raises(rsa.RSAError):
                    rsa.rsa_set_window_threads(h, bad)
            rsa.rsa_set_rounds_per_check(h, 1)
            rsa.rsa_set_rounds_per_check(h, 64)
            for bad in (0, 65):
                with pytest.raises(rsa.RSAError):
                    rsa.rsa_set_rounds_per_check(h, bad)
        finally:
            rsa.rsa_destroy(h)
