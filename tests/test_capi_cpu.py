"""The C-ABI library without a GPU: it loads, exports every declared entry
point, its host-only formulas match the oracle, and GPU entry points fail
cleanly when no device is present."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bem_create", "bem_solve", "bem_sweep", "bem_destroy", "bem_last_error",
                     "bem_convolve", "bem_influence_table", "bem_spectrum"):
        assert required in names


def test_library_exports_every_declared_symbol(bem_mod):
    lib = bem_mod.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("k", [-0.9, -0.45, 0.0, 0.3, 0.77])
@pytest.mark.parametrize("nu", [0.0, 0.3, 0.5])
def test_alpha_matches_oracle(bem_mod, oracle_mod, k, nu):
    assert bem_mod.alpha(k, nu) == pytest.approx(oracle_mod.alpha(k, nu), rel=1e-13)


def test_alpha_limits(bem_mod):
    # Boussinesq at k = 0 (any nu), Gibson's incompressible soil as k -> 1 at
    # nu = 0.5, where alpha / (1 - k) -> 1 / pi (a local, Winkler-type response),
    # and the purely radial stress field at nu = 1/(2+k)
    for nu in (0.0, 0.3, 0.5):
        assert bem_mod.alpha(0.0, nu) == pytest.approx(1.0 / math.pi, rel=1e-14)
    for k in (0.999, 0.9999):
        assert abs(math.pi * bem_mod.alpha(k, 0.5) / (1.0 - k) - 1.0) <= 1.0 - k
    # Frohlich-Holl radial-stress field at nu = 1/(2+k)
    for k in (0.1, 0.4, 0.8):
        assert bem_mod.alpha(k, 1.0 / (2.0 + k)) == pytest.approx(
            (2.0 + k) / (2.0 * math.pi * (1.0 + k) ** 2), rel=1e-13)


def test_alpha_invalid_is_nan(bem_mod):
    assert math.isnan(bem_mod.alpha(1.0, 0.3))
    assert math.isnan(bem_mod.alpha(0.2, 0.7))


def test_c1_corrected_matches_oracle_spline(bem_mod, oracle_mod):
    for k in np.linspace(-0.9, 0.9, 73):
        assert bem_mod.c1_corrected(float(k)) == pytest.approx(oracle_mod.c1_corrected(float(k)),
                                                               rel=1e-12)
    assert math.isnan(bem_mod.c1_corrected(0.95))


def test_table1_values_exact(bem_mod):
    from conftest import read_golden
    for k, c in read_golden("table1_c1.txt"):
        assert bem_mod.c1_corrected(k) == c


def test_p_crit_matches_oracle(bem_mod, oracle_mod):
    for k, nu, g, dl in [(0.3, 0.3, 1e-3, 1 / 2048), (-0.5, 0.25, 1e-2, 1 / 64), (0.65, 0.5, 1e-4, 0.01)]:
        assert bem_mod.p_crit(k, nu, g, dl) == pytest.approx(oracle_mod.p_crit(k, nu, g, dl), rel=1e-12)
    assert math.isnan(bem_mod.p_crit(0.3, 0.3, -1.0, 0.1))


def test_create_without_gpu_fails_cleanly(bem_mod):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bem_mod.BemError) as e:
        bem_mod.Handle(16, 16, 1 / 16, 1 / 16, 0.3, 0.3)
    assert e.value.code == bem_mod.BEM_ECUDA


def test_invalid_parameters_rejected_before_gpu(bem_mod):
    for args in [(1, 16, 0.1, 0.1, 0.3, 0.3), (16, 16, 0.1, 0.1, 1.0, 0.3),
                 (16, 16, 0.1, 0.1, 0.3, 0.6), (16, 16, -0.1, 0.1, 0.3, 0.3),
                 (5000, 16, 0.1, 0.1, 0.3, 0.3)]:
        with pytest.raises(bem_mod.BemError) as e:
            bem_mod.Handle(*args)
        assert e.value.code == bem_mod.BEM_EINVAL


def test_server_arguments_and_no_gpu(bem_mod):
    import torch
    for nworkers, budget in [(0, 1 << 30), (65, 1 << 30), (2, 1 << 20)]:
        with pytest.raises(bem_mod.BemError) as e:
            bem_mod.Server(nworkers, budget)
        assert e.value.code == bem_mod.BEM_EINVAL
    if not torch.cuda.is_available():
        with pytest.raises(bem_mod.BemError) as e:
            bem_mod.Server(2, 1 << 30)
        assert e.value.code == bem_mod.BEM_ECUDA


def test_server_footprint(bem_mod):
    f = bem_mod.Server.footprint
    assert f(1, 64) == 0 and f(64, 5000) == 0
    sizes = [f(n, n) for n in (16, 64, 256, 1024, 2048)]
    assert all(a < b for a, b in zip(sizes, sizes[1:]))
    # at least the FP32 and FP64 CG fields and the transposed half spectrum
    n = 1024
    assert f(n, n) > (4 + 8) * 5 * n * n + 16 * (n + 1) * n


def test_library_resolves_all_symbols_at_load(bem_mod):
    """Every internal symbol resolves when the library is loaded with immediate
    binding (an uninstantiated template would fail here, not at first call)."""
    import ctypes
    ctypes.CDLL(bem_mod.LIB_PATH, mode=os.RTLD_NOW)


def test_debug_checks_compile():
    """The bounds-checked kernels (-DBEM_DEBUG_CHECKS) compile; the debug build
    goes to its own directory, so it never replaces the release library."""
    import subprocess
    import tempfile
    from paper_1612_08395_gb300 import build as B
    assert B.DEBUG_LIB != B.LIB and os.path.dirname(B.DEBUG_LIB) != os.path.dirname(B.LIB)
    with tempfile.TemporaryDirectory() as d:
        for src in ("kern_f32_b.cu", "kern_f64_b.cu"):
            cmd = [B.nvcc(), *B.ARCH, *B.FLAGS, "-DBEM_DEBUG_CHECKS", "-c", os.path.join(B.CSRC, src),
                   "-o", os.path.join(d, src + ".o")]
            r = subprocess.run(cmd, capture_output=True, text=True)
            assert r.returncode == 0, r.stderr[-2000:]
