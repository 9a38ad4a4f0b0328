"""The C-ABI library loads on a machine without a GPU, exports every entry point that
include/*.h declares, and its structs have the layout the binding assumes. Only calls that
fail argument validation before touching CUDA are made here."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h")]
LIB = os.path.join(ROOT, "paper_1208_4830_gb300", "libsblm.so")


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(LIB):
        from paper_1208_4830_gb300 import build

        build.build()
    from paper_1208_4830_gb300 import sblm

    return sblm


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sblm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(LIB)
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(built.exported_symbols()) == names


def test_struct_layout_matches_header(built, tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sblm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(sblm_bounds), sizeof(sblm_ea_params),"
        " sizeof(sblm_ea_state), offsetof(sblm_ea_params, seed), offsetof(sblm_ea_state, best_genes),"
        " offsetof(sblm_ea_state, n_hist), offsetof(sblm_ea_params, n_islands),"
        " offsetof(sblm_ea_params, polish_radius)); return 0;}\n"
    )
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    s = built
    want = [
        ctypes.sizeof(s.Bounds),
        ctypes.sizeof(s.EAParams),
        ctypes.sizeof(s.EAState),
        s.EAParams.seed.offset,
        s.EAState.best_genes.offset,
        s.EAState.n_hist.offset,
        s.EAParams.n_islands.offset,
        s.EAParams.polish_radius.offset,
    ]
    assert got == want


def test_status_strings_and_defaults(built):
    lib = built._lib
    assert lib.sblm_status_str(0) == b"SBLM_OK"
    assert lib.sblm_status_str(1) == b"SBLM_EINVAL"
    p = built.params()
    # Appendix A defaults: N_pop = 1000, p_mut = 1%, N_tourn = ceil(N_pop/25), 10 generations, 1%
    assert (p.n_pop, p.p_mut0, p.n_tourn, p.stag_window, p.stag_rel, p.restart_after) == (1000, 0.01, 0, 10, 0.01, 10)


def test_argument_validation_without_gpu(built):
    lib = built._lib
    # negative sizes and unknown precision are rejected before any CUDA call
    assert lib.sblm_magnification(None, -1, None, 5, None, None, 0, None) == 1
    assert b"negative" in lib.sblm_last_error()
    assert lib.sblm_magnification(None, 3, None, 5, None, None, 9, None) == 1
    assert lib.sblm_chi2(None, 2, None, None, None, -4, None, 0, None) == 1
    p = built.params(n_pop=1)
    assert lib.sblm_ea_generation(None, None, 1, 6, ctypes.byref(p), 0, 0, None, None) == 1
    p = built.params(n_pop=64, stag_window=99)
    assert lib.sblm_ea_init(None, 64, 6, ctypes.byref(p), 0, None, None) == 1
    p = built.params(n_pop=64)
    assert lib.sblm_ea_init(None, 64, 17, ctypes.byref(p), 0, None, None) == 1
    b = built.bounds([0, 5, 0, 0, 0.3, -4], [0, 100, 1, 6, 3, 0])  # lo == hi for t0
    p = built.params(n_pop=64, n_gen=10)
    assert lib.sblm_fit(None, None, None, 10, ctypes.byref(b), ctypes.byref(p), None, None, None, None) == 1
    # the blended chi^2: negative sizes, an unknown precision, missing buffers
    assert lib.sblm_chi2_blend(None, -1, None, None, None, 5, None, None, 0, None) == 1
    assert lib.sblm_chi2_blend(None, 2, None, None, None, 5, None, None, 7, None) == 1
    assert lib.sblm_chi2_blend(None, 2, None, None, None, 5, None, None, 0, None) == 1
    assert b"NULL" in lib.sblm_last_error()
    # the single-lightcurve fitter takes neither the blend flag nor islands (batched fitters only)
    b = built.bounds([-20, 5, 0, 0, 0.3, -4], [20, 100, 1, 6, 3, 0])
    p = built.params(n_pop=64, n_gen=10, precision="mixed+blend")
    assert lib.sblm_fit(None, None, None, 10, ctypes.byref(b), ctypes.byref(p), None, None, None, None) == 1
    assert b"SBLM_BLEND" in lib.sblm_last_error()
    p = built.params(n_pop=64, n_gen=10, n_islands=2)
    assert lib.sblm_fit(None, None, None, 10, ctypes.byref(b), ctypes.byref(p), None, None, None, None) == 1
    assert b"islands" in lib.sblm_last_error()
    # zero-size work is a successful no-op
    assert lib.sblm_magnification(None, 0, None, 0, None, None, 0, None) == 0
    assert lib.sblm_chi2_blend(None, 0, None, None, None, 5, None, None, 0, None) == 0


def test_precision_strings():
    from paper_1208_4830_gb300 import sblm

    assert sblm._precision("fp64") == 0 and sblm._precision("mixed") == 1 and sblm._precision("fp32") == 2
    assert sblm._precision("mixed+blend") == 1 | sblm.BLEND and sblm._precision("fp64+blend") == sblm.BLEND
    assert sblm._precision(17) == 17
    with pytest.raises(ValueError):
        sblm._precision("mixed+islands")
    p = sblm.params()
    assert (p.n_islands, p.migration_interval) == (1, 20)


def test_binding_refuses_to_run_without_library(tmp_path):
    """The binding raises at import when libsblm.so is absent (no CPU fallback)."""
    import importlib.util

    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1208_4830_gb300", "sblm.py"), pkg / "sblm.py")
    spec = importlib.util.spec_from_file_location("sblm_nolib", pkg / "sblm.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_cnn_abi_layout_and_validation(built, tmp_path):
    from oracle import cnn as ocnn

    lib = built._lib
    assert built.cnn_num_params() == ocnn.N_PARAMS
    gcc = shutil.which("gcc")
    if gcc:
        src = tmp_path / "cnn_layout.c"
        src.write_text(
            '#include <stdio.h>\n#include <stddef.h>\n#include "sblm_cnn.h"\n'
            'int main(void){printf("%zu %zu %zu\\n", sizeof(sblm_cnn_train_params),'
            " offsetof(sblm_cnn_train_params, lr), offsetof(sblm_cnn_train_params, seed)); return 0;}\n"
        )
        exe = tmp_path / "cnn_layout"
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
        got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
        T = built.CnnTrainParams
        assert got == [ctypes.sizeof(T), T.lr.offset, T.seed.offset]
    p = built.cnn_train_params()
    assert (p.batch, p.n_steps, p.precision, p.lr, p.forced_frac) == (256, 4096, 2, 2e-3, 0.1)
    # rejected before any CUDA call
    assert lib.sblm_cnn_make_batch(0, 0, 0, 0.1, 1, None, None, None, None) == 1
    assert lib.sblm_cnn_make_batch(0, 0, 4, 1.5, 1, None, None, None, None) == 1
    assert lib.sblm_cnn_forward(None, None, 0, None, None) == 1
    assert lib.sblm_cnn_loss_grad(None, None, None, 4, None, None, None) == 1
    bad = built.cnn_train_params(batch=0)
    assert lib.sblm_cnn_train(None, None, ctypes.byref(bad), 0, 1, None, None) == 1
    bad = built.cnn_train_params(lr=-1.0)
    assert lib.sblm_cnn_adamw(None, None, None, ctypes.byref(bad), 1, None) == 1
    b = built.bounds([0, 5, 0, 0, 0.3, -4], [0, 100, 1, 6, 3, 0])
    assert lib.sblm_cnn_propose(None, None, 1, ctypes.byref(b), 4, 0, None, None) == 1
    assert lib.sblm_cnn_bin(None, None, None, None, 0, None, None, None) == 1
    pp = built.params(n_pop=64)
    assert lib.sblm_fit_batch_cnn(None, None, None, None, 1, None, ctypes.byref(pp), None, None, 2.0, None, None,
                                  None) == 1
